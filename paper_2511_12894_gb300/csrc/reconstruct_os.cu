// Overlap-save reconstruction (frequency form of the ratio identity, Eq. 7) with
// uniformly partitioned kernels, FP32.
//
// Block size B, partition length Lp = B / Q (Q = 2, 4 or 8) and hop H = B - Lp:
//   segment spectra (once per reference, shared by all neighbours), NQ = n / Lp of them
//     Zs[q] = FFT_B( z_ref[(q Lp + t) mod n], t < B )
//   kernel partition spectra (once per kernel set, FP64 then rounded)
//     C[j][p] = FFT_B( c_j[p Lp + u] for u < Lp, zero above ) / B,   p < P_j = ceil(L_j / Lp)
//   output block s of neighbour j (s < NB = ceil(n / H))
//     y = IFFT_B( sum_p Zs[(s (Q - 1) - p - 1) mod NQ] C[j][p] ),
//     w_j[s H + t - Lp] = y[t] for Lp <= t < B (and s H + t - Lp < n),
// which is w_j[i'] = sum_l c_j[l] z_ref[(i' - l) mod n] (the circular product of a B-point
// segment with a partition of Lp taps is free of wrap-around from t = Lp - 1 on), and
// z_j[i] = w_j[(i - m0_j) mod n]: the first lag is applied by relabelling outputs, so every
// neighbour shares Zs.  Real-form kernels have Hermitian partition spectra (C[B - k] =
// conj C[k]); their sets keep bins 0..B/2 only, in rows of B/2 + 8, and the product reads a
// bin above B/2 as the conjugate of its mirror (`herm`).  Q = 2 is the classic half-overlap form; larger Q keeps more outputs
// per block transform at the price of more (cheap) partition products.
// The window peaks are reduced per warp and merged across blocks with 64-bit
// atomicMax on (float bits of |z|^2) << 32 | (2^32 - 1 - i), which orders by value
// and then by the smallest index.
#include <algorithm>
#include <cmath>
#include <memory>

#include "os_tail.cuh"
#include "rf_internal.h"

namespace rf {

namespace {

template <int B>
__global__ void __launch_bounds__(B / 16) k_os_segments(const float2* __restrict__ z_ref, int64_t n, int Lp,
                                                        const float2* __restrict__ tw, float2* __restrict__ Zs) {
  using S = BlockFFTShape<B>;
  extern __shared__ float2 sm[];
  const int64_t s = blockIdx.x;
  const int tid = threadIdx.x;
  const int64_t mask = n - 1;
  float2 v[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) v[t] = z_ref[(s * Lp + tid + t * (B / 16)) & mask];
  block_fft<B, -1>(v, sm, tw);
  float2* out = Zs + s * B;
#pragma unroll
  for (int q = 0; q < 16 / S::RL; ++q)
#pragma unroll
    for (int t = 0; t < S::RL; ++t) out[tid + q * S::NT + t * (B / S::RL)] = v[q * S::RL + t];
}

// Segment spectra of several references: block (s, g) transforms segment s of z_refs[g].
template <int B>
__global__ void __launch_bounds__(B / 16) k_os_segments_batched(const float2* const* __restrict__ z_refs, int64_t n,
                                                                int Lp, const float2* __restrict__ tw,
                                                                float2* __restrict__ Zs_all) {
  using S = BlockFFTShape<B>;
  extern __shared__ float2 sm[];
  const int64_t s = blockIdx.x;
  const int64_t g = blockIdx.y;
  const int64_t NQ = n / Lp;
  const float2* z_ref = z_refs[g];
  const int tid = threadIdx.x;
  const int64_t mask = n - 1;
  float2 v[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) v[t] = z_ref[(s * Lp + tid + t * (B / 16)) & mask];
  block_fft<B, -1>(v, sm, tw);
  float2* out = Zs_all + (g * NQ + s) * B;
#pragma unroll
  for (int q = 0; q < 16 / S::RL; ++q)
#pragma unroll
    for (int t = 0; t < S::RL; ++t) out[tid + q * S::NT + t * (B / S::RL)] = v[q * S::RL + t];
}

// One neighbour's output blocks [s0, s1): spectral products, then the block tail (inverse block
// FFT and either the series (zrow != nullptr) or the window peaks (keys row kj)).
template <int B, int Q, bool WINMAX>
__device__ __forceinline__ void os_blocks(const float2* __restrict__ Zs, const float2* __restrict__ C, int P,
                                          int64_t m0, const float2* __restrict__ tw, int64_t n, int NQ, int s0,
                                          int s1, float2* __restrict__ zrow, unsigned long long* __restrict__ kj,
                                          int64_t W, int64_t nw, int fastwin, int herm, float2* sm) {
  static_assert(Q == 2 || Q == 4 || Q == 8, "partition ratio");
  const int tid = threadIdx.x;
  // partition spectrum loads: bins tid + t B/16; with the Hermitian half, the upper eight
  // (t >= 8, above B/2) come from the mirrors B/2 - tid - (t - 8) B/16, conjugated
  const int crow = os_row(B, herm != 0);
  const int hi_base = herm ? B / 2 - tid : B / 2 + tid;
  const int hi_step = herm ? -(B / 16) : B / 16;
  const float csgn = herm ? -1.f : 1.f;
  for (int s = s0; s < s1; ++s) {
    float2 v[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t] = make_float2(0.f, 0.f);
    // partitions outermost: each pass issues all 32 loads of the thread's bins at once.
    // The spectra stream through L2 only (ld.global.cg), so they do not evict the
    // twiddle tables from L1.
    int sp = s * (Q - 1) - 1;  // segment of partition 0; always < NQ
    for (int p = 0; p < P; ++p, --sp) {
      const int q = sp + ((sp < 0) ? NQ : 0);  // sp >= -NQ because P <= NQ
      const float2* zp = Zs + (int64_t)q * B + tid;
      const float2* cb = C + (int64_t)p * crow;
#pragma unroll
      for (int h = 0; h < 16; h += 8) {
        float2 z[8], c[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          z[t] = __ldcg(zp + (h + t) * (B / 16));
          c[t] = h == 0 ? __ldcg(cb + tid + t * (B / 16)) : __ldcg(cb + hi_base + t * hi_step);
        }
        if (h != 0) {
#pragma unroll
          for (int t = 0; t < 8; ++t) c[t].y *= csgn;
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          v[h + t].x = fmaf(z[t].x, c[t].x, fmaf(-z[t].y, c[t].y, v[h + t].x));
          v[h + t].y = fmaf(z[t].x, c[t].y, fmaf(z[t].y, c[t].x, v[h + t].y));
        }
      }
    }
    os_block_tail<B, Q, WINMAX>(v, s, m0, n, zrow, kj, W, nw, fastwin, tw, sm);
  }
}

// Neighbours idx[y0 + blockIdx.y] of one layout bucket; blockIdx.x takes SC output blocks.
template <int B, int Q, bool WINMAX>
__global__ void __launch_bounds__(B / 16, 16384 / B) k_os(const float2* __restrict__ Zs, const float2* __restrict__ Cs,
                                              const int64_t* __restrict__ spec_off, const int* __restrict__ parts,
                                              const int* __restrict__ lag0, const int* __restrict__ idx, int y0,
                                              const float2* __restrict__ tw, int64_t n,
                                              int NQ, int NB, int SC, float2* __restrict__ z_out,
                                              unsigned long long* __restrict__ keys, int64_t W, int64_t nw,
                                              int fastwin, int herm) {
  extern __shared__ float2 sm[];
  const int j = idx[y0 + blockIdx.y];
  const int s0 = blockIdx.x * SC;
  const int s1 = min(NB, s0 + SC);
  os_blocks<B, Q, WINMAX>(Zs, Cs + spec_off[j], parts[j], lag0[j], tw, n, NQ, s0, s1,
                       WINMAX ? nullptr : z_out + (int64_t)j * n, WINMAX ? keys + (int64_t)j * nw : nullptr, W, nw,
                       fastwin, herm, sm);
}

// Batched form: neighbours of several references in one persistent launch.  Each item
// describes one neighbour (its partition spectra, partitions, first lag, the segment
// spectra of its reference and its output row); work units are (item, chunk of SC
// output blocks), claimed in the order of `order` (unit code item * nchunk + chunk) from
// an atomic counter.  The host orders them by reference, then by tiles of output chunks x
// neighbours, so the segment spectra a tile reads and its neighbours' partition spectra stay
// in L2 while the tile's units run (a 2^23-sample reference has 134-268 MB of segment
// spectra, more than L2 holds).

template <int B, int Q>
__global__ void __launch_bounds__(B / 16, 16384 / B) k_os_batched(const OsItem* __restrict__ items,
                                                                 const long long* __restrict__ order, int64_t units,
                                                                 int nchunk, const float2* __restrict__ tw, int64_t n,
                                                                 int NQ, int NB, int SC,
                                                                 unsigned long long* __restrict__ keys,
                                                                 int64_t W, int64_t nw, int fastwin, int herm,
                                                                 unsigned long long* __restrict__ counter) {
  extern __shared__ float2 sm[];
  __shared__ long long s_unit;
  for (;;) {
    if (threadIdx.x == 0) s_unit = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const long long u = s_unit;
    __syncthreads();
    if (u >= units) break;
    const long long code = order[u];
    const OsItem it = items[code / nchunk];
    const int s0 = (int)(code % nchunk) * SC;
    const int s1 = min(NB, s0 + SC);
    os_blocks<B, Q, true>(it.Zs, it.C, it.P, it.lag0, tw, n, NQ, s0, s1, nullptr, keys + it.row * nw, W, nw, fastwin,
                          herm, sm);
  }
}

__global__ void k_unpack_keys(const unsigned long long* __restrict__ keys, int64_t count, float* __restrict__ mx,
                              int* __restrict__ arg) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const unsigned long long k = keys[i];
  mx[i] = __uint_as_float((unsigned int)(k >> 32));
  arg[i] = (int)(0xffffffffu - (unsigned int)(k & 0xffffffffull));
}

// rows[g][u] = taps of partition (j, p) = g, promoted to FP64, zero from u = Lp or l = L_j on
// (taps: float2, or float for a real-form set)
__global__ void k_os_fill(const void* __restrict__ taps, int real, const int64_t* __restrict__ off,
                          const int* __restrict__ len, const int* __restrict__ gj, const int* __restrict__ gp,
                          int B, int Lp, double2* __restrict__ rows) {
  const int g = blockIdx.y;
  const int j = gj[g], p = gp[g];
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < B; u += gridDim.x * blockDim.x) {
    double2 v = make_double2(0.0, 0.0);
    const int64_t l = (int64_t)p * Lp + u;
    if (u < Lp && l < len[j]) {
      if (real) {
        v = make_double2((double)static_cast<const float*>(taps)[off[j] + l], 0.0);
      } else {
        const float2 c = static_cast<const float2*>(taps)[off[j] + l];
        v = make_double2((double)c.x, (double)c.y);
      }
    }
    rows[(int64_t)g * B + u] = v;
  }
}

__global__ void k_os_round(const double2* __restrict__ spec, int64_t count, double scale, float2* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = make_float2((float)(spec[i].x * scale), (float)(spec[i].y * scale));
}

// Hermitian half of `rows` B-point spectra of real partitions: bins 0..B/2 into rows of
// B/2 + 8 (the pad zero); bins 0 and B/2 are real, so their imaginary rounding noise is dropped.
__global__ void k_os_round_half(const double2* __restrict__ spec, int rows, int B, double scale,
                                float2* __restrict__ out) {
  const int rs = B / 2 + 8;
  const int64_t count = (int64_t)rows * rs;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int64_t g = i / rs;
  const int k = (int)(i - g * rs);
  float2 v = make_float2(0.f, 0.f);
  if (k <= B / 2) {
    const double2 c = spec[g * B + k];
    v = make_float2((float)(c.x * scale), (k == 0 || k == B / 2) ? 0.f : (float)(c.y * scale));
  }
  out[i] = v;
}

// 32768-point blocks on CTA pairs: the layout, the cluster helpers and the block tail are in
// os_tail.cuh.

// Segment spectra of the B2 layout (no cluster needed): block (q, r, g) transforms
//   u_0[m] = x[m] + x[m + BH],  u_1[m] = (x[m] - x[m + BH]) exp(-2 pi i m / B2),
// x[m] = z_ref_g[(q Lp + m) mod n], giving the bins of parity r (decimation in frequency).
__global__ void __launch_bounds__(kBH / 16) k_os2_segments(const float2* __restrict__ z_one,
                                                          const float2* const* __restrict__ z_many, int64_t n, int Lp,
                                                          int NQ, const float2* __restrict__ tw,
                                                          const float2* __restrict__ twc, float2* __restrict__ Zs_all) {
  using S = BlockFFTShape<kBH>;
  extern __shared__ float2 sm[];
  const int64_t q = blockIdx.x;
  const int r = blockIdx.y;
  const int64_t g = blockIdx.z;
  const float2* z = z_many ? z_many[g] : z_one;
  const int tid = threadIdx.x;
  const int64_t mask = n - 1;
  float2 v[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    const int m = tid + t * S::NT;
    const float2 a = z[(q * Lp + m) & mask];
    const float2 b = z[(q * Lp + m + kBH) & mask];
    v[t] = r == 0 ? cadd(a, b) : cmul(csub(a, b), __ldg(twc + m));
  }
  block_fft<kBH, -1>(v, sm, tw);
  float2* out = Zs_all + ((int64_t)g * NQ + q) * kB2 + (int64_t)r * kBH;
#pragma unroll
  for (int qq = 0; qq < 16 / S::RL; ++qq)
#pragma unroll
    for (int t = 0; t < S::RL; ++t) out[tid + qq * S::NT + t * (kBH / S::RL)] = v[qq * S::RL + t];
}

// Spectral products of one output block for the bins of parity r (as os_blocks, on the
// parity-split spectra).
template <int Q>
__device__ __forceinline__ void os2_products(float2 (&v)[16], const float2* __restrict__ Zs,
                                             const float2* __restrict__ C, int P, int NQ, int s, unsigned r, int tid) {
  constexpr int NT = kBH / 16;
#pragma unroll
  for (int t = 0; t < 16; ++t) v[t] = make_float2(0.f, 0.f);
  int sp = s * (Q - 1) - 1;  // segment of partition 0; always < NQ
  for (int p = 0; p < P; ++p, --sp) {
    const int q = sp + ((sp < 0) ? NQ : 0);  // sp >= -NQ because P <= NQ
    const float2* zp = Zs + (int64_t)q * kB2 + (int64_t)r * kBH + tid;
    const float2* cp = C + (int64_t)p * kB2 + (int64_t)r * kBH + tid;
#pragma unroll
    for (int h = 0; h < 16; h += 8) {
      float2 z[8], c[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        z[t] = __ldcg(zp + (h + t) * NT);
        c[t] = __ldcg(cp + (h + t) * NT);
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        v[h + t].x = fmaf(z[t].x, c[t].x, fmaf(-z[t].y, c[t].y, v[h + t].x));
        v[h + t].y = fmaf(z[t].x, c[t].y, fmaf(z[t].y, c[t].x, v[h + t].y));
      }
    }
  }
}

// Output blocks [s0, s1) of one neighbour on a CTA pair: per block, this CTA's parity half of
// the spectral products, then the pair's block tail (os_tail.cuh).
// Zs: the reference's segment spectra [NQ][B2]; C: the neighbour's partition spectra [P][B2],
// both parity-split.
template <int Q, bool WINMAX>
__device__ __forceinline__ void os2_blocks(const float2* __restrict__ Zs, const float2* __restrict__ C, int P,
                                           int64_t m0, const float2* __restrict__ tw, const float2* __restrict__ twc,
                                           int64_t n, int NQ, int s0, int s1, float2* __restrict__ zrow,
                                           unsigned long long* __restrict__ kj, int64_t W, int64_t nw, int fastwin,
                                           float2* sm) {
  static_assert(Q == 2 || Q == 4, "partition ratio");
  const unsigned r = cluster_rank();
  const uint32_t peer = cluster_peer_addr(sm, r ^ 1u);
  const int tid = threadIdx.x;
  for (int s = s0; s < s1; ++s) {
    float2 v[16];
    os2_products<Q>(v, Zs, C, P, NQ, s, r, tid);
    os2_block_tail<Q, WINMAX>(v, s, m0, n, zrow, kj, W, nw, fastwin, tw, twc, sm, r, peer);
  }
}

template <int Q, bool WINMAX>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kBH / 16, 1)
    k_os2(const float2* __restrict__ Zs, const float2* __restrict__ Cs, const int64_t* __restrict__ spec_off,
          const int* __restrict__ parts, const int* __restrict__ lag0, const int* __restrict__ idx, int y0,
          const float2* __restrict__ tw, const float2* __restrict__ twc, int64_t n, int NQ, int NB, int SC,
          float2* __restrict__ z_out, unsigned long long* __restrict__ keys, int64_t W, int64_t nw, int fastwin) {
  extern __shared__ float2 sm[];
  const int j = idx[y0 + blockIdx.y];
  const int s0 = (int)(blockIdx.x >> 1) * SC;
  const int s1 = min(NB, s0 + SC);
  os2_blocks<Q, WINMAX>(Zs, Cs + spec_off[j], parts[j], lag0[j], tw, twc, n, NQ, s0, s1,
                        WINMAX ? nullptr : z_out + (int64_t)j * n, WINMAX ? keys + (int64_t)j * nw : nullptr, W, nw,
                        fastwin, sm);
}

// Batched form: cluster (chunk, item) of a grid of (2 nchunk, count) CTAs.
template <int Q>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kBH / 16, 1)
    k_os2_batched(const OsItem* __restrict__ items, int nchunk, const float2* __restrict__ tw,
                  const float2* __restrict__ twc, int64_t n, int NQ, int NB, int SC,
                  unsigned long long* __restrict__ keys, int64_t W, int64_t nw, int fastwin) {
  extern __shared__ float2 sm[];
  const OsItem it = items[blockIdx.y];
  const int s0 = (int)(blockIdx.x >> 1) * SC;
  const int s1 = min(NB, s0 + SC);
  os2_blocks<Q, true>(it.Zs, it.C, it.P, it.lag0, tw, twc, n, NQ, s0, s1, nullptr, keys + it.row * nw, W, nw, fastwin,
                      sm);
}

// partition spectra of the B2 layout: rows of B2 bins, rounded and stored parity-split
__global__ void k_os2_round(const double2* __restrict__ spec, int64_t count, double scale, float2* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int k = (int)(i & (kB2 - 1));
  out[(i - k) + (k & 1) * kBH + (k >> 1)] = make_float2((float)(spec[i].x * scale), (float)(spec[i].y * scale));
}


template <int B>
size_t os_smem() {
  return sizeof(float2) * BlockFFTShape<B>::SMEM;
}

template <int B>
void launch_os_segments(rf_ctx* c, const float2* z_ref, int Lp, float2* Zs, cudaStream_t s) {
  const int NQ = (int)(c->n / Lp);
  const float2* tw = c->twb32.as<float2>() + c->twb_off[BlockFFTShape<B>::LOGB];
  auto fn = k_os_segments<B>;
  RF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)os_smem<B>()));
  fn<<<NQ, B / 16, os_smem<B>(), s>>>(z_ref, c->n, Lp, tw, Zs);
  RF_LAUNCHED();
}

// outputs of a window that one warp's epilogue covers (32 threads x H / (B / 16) outputs)
template <int B, int Q>
constexpr int os_warp_span() {
  return 32 * ((B - B / Q) / (B / 16));
}

template <int B, int Q, bool WINMAX>
void launch_os(rf_ctx* c, const rf_kernels* kern, const OsBucket& bk, const float2* Zs, float2* z_out,
               unsigned long long* keys, int64_t W, cudaStream_t s) {
  constexpr int Lp = B / Q, H = B - Lp;
  const int NQ = (int)(c->n / Lp);
  const int NB = (int)((c->n + H - 1) / H);
  const int count = (int)bk.idx.size();
  const float2* tw = c->twb32.as<float2>() + c->twb_off[BlockFFTShape<B>::LOGB];
  const int64_t nw = WINMAX ? (c->n + W - 1) / W : 0;
  // output blocks per CTA: enough CTAs for every SM several times over
  int SC = 8;
  while (SC > 1 && (int64_t)count * ((NB + SC - 1) / SC) < 8LL * c->nsm) SC /= 2;
  const int nchunk = (NB + SC - 1) / SC;
  const int fastwin = (WINMAX && W >= os_warp_span<B, Q>()) ? 1 : 0;  // a warp's outputs span <= 2 windows
  auto fn = k_os<B, Q, WINMAX>;
  RF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)os_smem<B>()));
  for (int done = 0; done < count; done += 65535) {
    const int cnt = std::min(65535, count - done);
    dim3 grid((unsigned)nchunk, (unsigned)cnt);
    fn<<<grid, B / 16, os_smem<B>(), s>>>(Zs, kern->os_spec.as<float2>(), kern->os_off_d.as<int64_t>(),
                                          kern->os_parts_d.as<int>(), kern->lag0_d.as<int>(), bk.idx_d.as<int>(), done,
                                          tw, c->n, NQ, NB, SC, z_out, keys, W, nw, fastwin, kern->real ? 1 : 0);
    RF_LAUNCHED();
  }
}

// dynamic shared memory of the pair kernels: the 16384-point transform plus two 8192-float
// |y|^2 staging rows
size_t os2_smem() { return os2_tail_smem(); }

// Segment spectra of the pair layout for one reference (z_many == nullptr) or G of them.
void launch_os2_segments(rf_ctx* c, const float2* z_one, const float2* const* z_many, int G, int Lp, float2* Zs,
                         cudaStream_t s) {
  const int NQ = (int)(c->n / Lp);
  const float2* tw = c->twb32.as<float2>() + c->twb_off[14];
  const float2* twc = c->twb32.as<float2>() + c->twb_off[15];
  RF_REQUIRE(G <= 65535, "at most 65535 references per batch");
  RF_CUDA(cudaFuncSetAttribute(k_os2_segments, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)os_smem<kBH>()));
  k_os2_segments<<<dim3((unsigned)NQ, 2, (unsigned)G), kBH / 16, os_smem<kBH>(), s>>>(z_one, z_many, c->n, Lp, NQ, tw,
                                                                                      twc, Zs);
  RF_LAUNCHED();
}

// One layout bucket on CTA pairs: clusters (chunk of SC output blocks, neighbour).
template <int Q, bool WINMAX>
void launch_os2(rf_ctx* c, const rf_kernels* kern, const OsBucket& bk, const float2* Zs, float2* z_out,
                unsigned long long* keys, int64_t W, cudaStream_t s) {
  constexpr int Lp = kB2 / Q, H = kB2 - Lp;
  const int NQ = (int)(c->n / Lp);
  const int NB = (int)((c->n + H - 1) / H);
  const int count = (int)bk.idx.size();
  const float2* tw = c->twb32.as<float2>() + c->twb_off[14];
  const float2* twc = c->twb32.as<float2>() + c->twb_off[15];
  const int64_t nw = WINMAX ? (c->n + W - 1) / W : 0;
  // output blocks per cluster: enough clusters for every SM pair several times over
  int SC = 8;
  while (SC > 1 && (int64_t)count * ((NB + SC - 1) / SC) < 4LL * c->nsm) SC /= 2;
  const int nchunk = (NB + SC - 1) / SC;
  const int fastwin = (WINMAX && W >= 256) ? 1 : 0;  // a warp's 256 outputs of a run span <= 2 windows
  auto fn = k_os2<Q, WINMAX>;
  RF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)os2_smem()));
  for (int done = 0; done < count; done += 65535) {
    const int cnt = std::min(65535, count - done);
    dim3 grid((unsigned)(2 * nchunk), (unsigned)cnt);
    fn<<<grid, kBH / 16, os2_smem(), s>>>(Zs, kern->os_spec.as<float2>(), kern->os_off_d.as<int64_t>(),
                                              kern->os_parts_d.as<int>(), kern->lag0_d.as<int>(), bk.idx_d.as<int>(),
                                              done, tw, twc, c->n, NQ, NB, SC, z_out, keys, W, nw, fastwin);
    RF_LAUNCHED();
  }
}

template <typename F>
void dispatch_b(int B, F&& f) {
  switch (B) {
    case 512: f(std::integral_constant<int, 512>{}); break;
    case 1024: f(std::integral_constant<int, 1024>{}); break;
    case 2048: f(std::integral_constant<int, 2048>{}); break;
    case 4096: f(std::integral_constant<int, 4096>{}); break;
    case 8192: f(std::integral_constant<int, 8192>{}); break;
    case 16384: f(std::integral_constant<int, 16384>{}); break;
    default: RF_REQUIRE(false, "overlap-save block size %d is not supported", B);
  }
}

template <typename F>
void dispatch_bq(int B, int Q, F&& f) {
  dispatch_b(B, [&](auto bc) {
    switch (Q) {
      case 2: f(bc, std::integral_constant<int, 2>{}); break;
      case 4: f(bc, std::integral_constant<int, 4>{}); break;
      case 8: f(bc, std::integral_constant<int, 8>{}); break;
      default: RF_REQUIRE(false, "overlap-save partition ratio %d is not supported", Q);
    }
  });
}

}  // namespace

namespace {

// Stage tables of one block size, in the order block_fft reads them.
template <int B>
void append_tables(std::vector<float2>& out) {
  using S = BlockFFTShape<B>;
  const size_t start = out.size();
  int Ns = 16;
  for (int st = 0; st < block_mid_stages<B>(); ++st) {
    const std::vector<double2> w = host_twiddles(16 * (int64_t)Ns);  // exp(-2 pi i m / (16 Ns))
    for (int t = 0; t < 16; ++t)
      for (int k = 0; k < Ns; ++k) {
        const double2 v = w[(size_t)t * k];
        out.push_back(make_float2((float)v.x, (float)v.y));
      }
    Ns *= 16;
  }
  const std::vector<double2> w = host_twiddles(B);  // last stage: exp(-2 pi i t b / B)
  for (int t = 0; t < S::RL; ++t)
    for (int b = 0; b < B / S::RL; ++b) {
      const double2 v = w[(size_t)t * b];
      out.push_back(make_float2((float)v.x, (float)v.y));
    }
  if (out.size() - start != (size_t)block_table_size<B>()) throw Fail{RF_EINVAL};
}

}  // namespace

std::vector<float2> block_fft_tables(int64_t off[16]) {
  std::vector<float2> out;
  for (int b = 0; b < 16; ++b) off[b] = 0;
  off[9] = (int64_t)out.size();
  append_tables<512>(out);
  off[10] = (int64_t)out.size();
  append_tables<1024>(out);
  off[11] = (int64_t)out.size();
  append_tables<2048>(out);
  off[12] = (int64_t)out.size();
  append_tables<4096>(out);
  off[13] = (int64_t)out.size();
  append_tables<8192>(out);
  off[14] = (int64_t)out.size();
  append_tables<16384>(out);
  // the pair layout's twiddles exp(-2 pi i m / 32768), m < 16384 (segment split and combine)
  off[15] = (int64_t)out.size();
  {
    const std::vector<double2> w = host_twiddles(kB2);
    for (int m = 0; m < kBH; ++m) out.push_back(make_float2((float)w[(size_t)m].x, (float)w[(size_t)m].y));
  }
  return out;
}

// Layout choice by a cost model.  Per neighbour, a layout (B, Lp) runs NB = ceil(n / (B - Lp))
// output blocks, each one inverse block transform plus P = ceil(L / Lp) spectral
// multiply-adds; the model charges F(B) + P M(B) per block, with F and M the throughput
// costs per block (ns, whole GPU) measured on a GB300 for B >= 4096 on the 3.5PN
// 2^20-sample workload and scaled by B log B (F) and B (M) below that, and a fill penalty
// when the launch has fewer blocks than the GPU holds at once.
double os_layout_cost(const rf_ctx* c, const std::vector<int>& lengths, int B, int Lp) {
  // B = 512 .. 32768; the 32768-point block runs on a CTA pair (two 16384-point transforms
  // plus the exchange, estimated)
  static const double F[7] = {0.9, 1.9, 4.2, 9.9, 29.5, 70.3, 155.0};
  static const double M[7] = {0.37, 0.73, 1.47, 2.93, 5.1, 10.8, 21.6};
  int b = 0;
  while ((512 << b) < B) ++b;
  const int64_t H = B - Lp;
  const int64_t NB = (c->n + H - 1) / H;
  double cost = 0.0;
  for (const int L : lengths) cost += (double)NB * (F[b] + (double)std::max(1, (L + Lp - 1) / Lp) * M[b]);
  const double blocks = (double)NB * (double)lengths.size();
  const double slots = B > 16384 ? (double)c->nsm / 2 : (double)c->nsm * (16384 / B);
  return blocks < slots ? cost * slots / blocks : cost;
}

void os_choose_layout(const rf_ctx* c, const std::vector<int>& lengths, int block, bool real, int* B_out,
                      int* Lp_out) {
  double best = 0.0;
  int bB = 0, bL = 0;
  for (int B = 512; B <= kB2; B *= 2) {
    if (B > c->n || (block && B != block) || (real && B == kB2)) continue;
    for (int Q = 2; Q <= (B == kB2 ? 4 : 8); Q *= 2) {
      const double cost = os_layout_cost(c, lengths, B, B / Q);
      if (!bB || cost < best) {
        best = cost;
        bB = B;
        bL = B / Q;
      }
    }
  }
  RF_REQUIRE(bB, "no overlap-save layout for block %d and n=%lld", block, (long long)c->n);
  *B_out = bB;
  *Lp_out = bL;
}

static void check_layout(const rf_ctx* c, int B, int Lp, bool real) {
  RF_REQUIRE(B >= 512 && B <= kB2 && (B & (B - 1)) == 0 && B <= c->n, "overlap-save block %d invalid for n=%lld", B,
             (long long)c->n);
  RF_REQUIRE(!real || B < kB2, "real-form kernels take overlap-save blocks of at most %d points", kB2 / 2);
  RF_REQUIRE(Lp == B / 2 || Lp == B / 4 || (Lp == B / 8 && B < kB2),
             "overlap-save partition length %d must be B/2, B/4 or (below 32768) B/8", Lp);
}

// ---------------------------------------------------------------- buckets of other forms

// Kernel set of the neighbours idx of `kern` (taps copied), for a bucket that runs the direct
// or tensor-core form.
std::shared_ptr<rf_kernels> make_subset(const rf_kernels* kern, const std::vector<int32_t>& idx, cudaStream_t s) {
  std::shared_ptr<rf_kernels> sub(new rf_kernels());
  const int k = (int)idx.size();
  sub->k = k;
  sub->n = kern->n;
  sub->dtype = kern->dtype;
  sub->real = kern->real;
  sub->offset.assign((size_t)k + 1, 0);
  for (int q = 0; q < k; ++q) {
    const int j = idx[q];
    sub->len.push_back(kern->len[j]);
    sub->lag0.push_back(kern->lag0[j]);
    sub->df_low.push_back(kern->df_low[j]);
    sub->grid.push_back(kern->grid[j]);
    sub->offset[q + 1] = sub->offset[q] + kern->len[j];
  }
  sub->max_len = k ? *std::max_element(sub->len.begin(), sub->len.end()) : 0;
  const size_t esz = tap_bytes(kern);
  sub->taps.ensure(std::max<size_t>(16, (size_t)sub->offset[k] * esz));
  for (int q = 0; q < k; ++q)
    if (sub->len[q])
      RF_CUDA(cudaMemcpyAsync(static_cast<char*>(sub->taps.p) + sub->offset[q] * esz,
                              static_cast<const char*>(kern->taps.p) + kern->offset[idx[q]] * esz,
                              (size_t)sub->len[q] * esz, cudaMemcpyDeviceToDevice, s));
  sub->len_d.ensure(std::max<size_t>(16, sizeof(int32_t) * k));
  sub->lag0_d.ensure(std::max<size_t>(16, sizeof(int32_t) * k));
  sub->off_d.ensure(sizeof(int64_t) * (k + 1));
  if (k) {
    RF_CUDA(cudaMemcpyAsync(sub->len_d.p, sub->len.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, s));
    RF_CUDA(cudaMemcpyAsync(sub->lag0_d.p, sub->lag0.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, s));
  }
  RF_CUDA(cudaMemcpyAsync(sub->off_d.p, sub->offset.data(), sizeof(int64_t) * (k + 1), cudaMemcpyHostToDevice, s));
  RF_CUDA(cudaStreamSynchronize(s));  // the host vectors are read by the copies above
  return sub;
}

__global__ void k_scatter_peaks(const float* __restrict__ P, const int* __restrict__ A, int rows, int64_t nw,
                                const int* __restrict__ idx, int64_t row0, float* __restrict__ max_out,
                                int* __restrict__ arg_out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)rows * nw) return;
  const int64_t r = i / nw, w = i - r * nw;
  const int64_t d = (row0 + idx[r]) * nw + w;
  max_out[d] = P[i];
  arg_out[d] = A[i];
}

template <typename V>
__global__ void k_scatter_series(const V* __restrict__ src, int rows, int64_t n, const int* __restrict__ idx,
                                 V* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)rows * n) return;
  const int64_t r = i / n, t = i - r * n;
  dst[(int64_t)idx[r] * n + t] = src[i];
}

// Rows of a direct or tensor-core bucket: its subset runs into a temporary, whose rows go to
// rows row0 + idx of the window peaks (or of the series z_out).
void run_bucket_form(rf_ctx* c, const void* z_ref, const OsBucket& bk, int64_t W, float* max_out,
                     int32_t* argmax_out, void* z_out, int64_t row0, cudaStream_t s) {
  rf_kernels* sub = bk.sub.get();
  const int rows = sub ? sub->k : 0;
  if (!rows) return;
  const int64_t n = c->n;
  if (max_out) {
    const int64_t nw = (n + W - 1) / W;
    c->mix_tmp.ensure((sizeof(float) + sizeof(int32_t)) * (size_t)rows * nw + 256);
    float* P = c->mix_tmp.as<float>();
    int32_t* A = reinterpret_cast<int32_t*>(P + (int64_t)rows * nw);
    if (bk.algo == RF_ALGO_GEMM) reconstruct_gemm(c, z_ref, sub, bk.prec, nullptr, W, P, A, s);
    else reconstruct_direct(c, z_ref, sub, nullptr, W, P, A, s);
    const int64_t count = (int64_t)rows * nw;
    k_scatter_peaks<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(P, A, rows, nw, bk.idx_d.as<int>(), row0,
                                                                     max_out, argmax_out);
    RF_LAUNCHED();
  } else {
    c->mix_tmp.ensure(sizeof(float2) * (size_t)rows * n + 256);
    float2* zt = c->mix_tmp.as<float2>();
    if (bk.algo == RF_ALGO_GEMM) reconstruct_gemm(c, z_ref, sub, bk.prec, zt, 0, nullptr, nullptr, s);
    else reconstruct_direct(c, z_ref, sub, zt, 0, nullptr, nullptr, s);
    const int64_t count = (int64_t)rows * n;
    k_scatter_series<float2><<<(unsigned)((count + 255) / 256), 256, 0, s>>>(
        zt, rows, n, bk.idx_d.as<int>(), static_cast<float2*>(z_out) + row0 * n);
    RF_LAUNCHED();
  }
}

void os_prepare_buckets(rf_ctx* c, rf_kernels* kern, int nb, const int32_t* cuts, const int32_t* Bs,
                        const int32_t* Lps, cudaStream_t s) {
  RF_REQUIRE(nb >= 1 && nb <= 8, "between 1 and 8 layout buckets");
  std::vector<BucketSpec> spec(nb);
  for (int b = 0; b < nb; ++b) spec[b] = BucketSpec{cuts[b], RF_ALGO_OS, RF_PREC_NATIVE, Bs[b], Lps[b]};
  os_prepare_forms(c, kern, nb, spec.data(), s);
}

void os_prepare_forms(rf_ctx* c, rf_kernels* kern, int nb, const BucketSpec* spec, cudaStream_t s) {
  RF_REQUIRE(kern->dtype == RF_F32, "overlap-save needs the FP32 grid");
  RF_REQUIRE(nb >= 1 && nb <= 8, "between 1 and 8 layout buckets");
  RF_REQUIRE(spec[0].cut == 0, "the first bucket starts at length 0");
  for (int b = 0; b < nb; ++b) {
    const BucketSpec& o = spec[b];
    RF_REQUIRE(b == 0 || o.cut > spec[b - 1].cut, "bucket cuts must increase");
    if (o.algo == RF_ALGO_OS) {
      check_layout(c, o.block, o.part, kern->real);
    } else if (o.algo == RF_ALGO_OS_BINS) {
      check_layout(c, o.block, o.part, kern->real);
      RF_REQUIRE(bins_layout_ok(o.block, o.part),
                 "two-phase overlap-save takes B in {4096, 8192, 16384} with Lp = B/2 or B/4, or B = 32768 with "
                 "Lp = 16384 (got %d, %d)", o.block, o.part);
    } else if (o.algo == RF_ALGO_GEMM) {
      RF_REQUIRE(o.prec >= RF_PREC_BF16 && o.prec <= RF_PREC_3XTF32, "a tensor-core bucket needs a split precision");
      RF_REQUIRE(c->n % 128 == 0, "the tensor-core form needs n to be a multiple of 128");
      RF_REQUIRE(gemm_layout_ok(o.prec, o.block, o.part),
                 "tensor-core layout (%d neighbours, %d tiles) is not one of (16, %d), (%d, 1), (0, 0)", o.block,
                 o.part, gemm_stacked_shifts(o.prec), gemm_wide_nj(o.prec));
    } else {
      RF_REQUIRE(o.algo == RF_ALGO_DIRECT, "bucket %d: unknown form %d", b, o.algo);
    }
  }
  if (kern->os_ready && (int)kern->os_buckets.size() == nb) {
    bool same = true;
    for (int b = 0; b < nb; ++b) {
      const OsBucket& o = kern->os_buckets[b];
      const BucketSpec& q = spec[b];
      same = same && o.cut_lo == q.cut && o.algo == q.algo &&
             ((q.algo == RF_ALGO_OS || q.algo == RF_ALGO_OS_BINS) ? (o.B == q.block && o.Lp == q.part)
                                   : (q.algo != RF_ALGO_GEMM ||
                                      (o.prec == q.prec && o.gemm_nj == q.block && o.gemm_s == q.part)));
    }
    if (same) return;
  }
  const int k = kern->k;
  std::vector<OsBucket> bk(nb);
  for (int b = 0; b < nb; ++b) {
    bk[b].cut_lo = spec[b].cut;
    bk[b].algo = spec[b].algo;
    if (spec[b].algo == RF_ALGO_OS || spec[b].algo == RF_ALGO_OS_BINS) {
      bk[b].B = spec[b].block;
      bk[b].Lp = spec[b].part;
    } else if (spec[b].algo == RF_ALGO_GEMM) {
      bk[b].prec = spec[b].prec;
      bk[b].gemm_nj = spec[b].block;
      bk[b].gemm_s = spec[b].part;
    }
  }
  std::vector<int> bucket_of(k);
  for (int j = 0; j < k; ++j) {
    int b = nb - 1;
    while (b > 0 && kern->len[j] < spec[b].cut) --b;
    bucket_of[j] = b;
    bk[b].idx.push_back(j);
  }
  for (int b = 0; b < nb; ++b)
    if (bk[b].algo == RF_ALGO_GEMM)
      for (const int j : bk[b].idx)
        RF_REQUIRE(kern->len[j] <= gemm_max_len(), "a tensor-core bucket takes kernels of at most %d taps",
                   gemm_max_len());
  // spectra bucket after bucket (overlap-save buckets only), kernels in index order inside a bucket
  std::vector<int> parts(k, 0);
  std::vector<int64_t> off(k, 0);
  int64_t total = 0;
  for (int b = 0; b < nb; ++b) {
    if (bk[b].algo != RF_ALGO_OS && bk[b].algo != RF_ALGO_OS_BINS) continue;
    for (const int j : bk[b].idx) {
      parts[j] = std::max(1, (kern->len[j] + bk[b].Lp - 1) / bk[b].Lp);
      off[j] = total;
      total += (int64_t)parts[j] * os_row(bk[b].B, kern->real);
    }
  }
  kern->os_ready = false;
  kern->os_spec.ensure(std::max<size_t>(16, sizeof(float2) * (size_t)total));
  kern->os_off_d.ensure(std::max<size_t>(16, sizeof(int64_t) * k));
  kern->os_parts_d.ensure(std::max<size_t>(16, sizeof(int) * k));
  if (k) {
    RF_CUDA(cudaMemcpyAsync(kern->os_off_d.p, off.data(), sizeof(int64_t) * k, cudaMemcpyHostToDevice, s));
    RF_CUDA(cudaMemcpyAsync(kern->os_parts_d.p, parts.data(), sizeof(int) * k, cudaMemcpyHostToDevice, s));
  }
  for (int b = 0; b < nb; ++b) {
    OsBucket& o = bk[b];
    o.idx_d.ensure(std::max<size_t>(16, sizeof(int32_t) * o.idx.size()));
    if (!o.idx.empty())
      RF_CUDA(cudaMemcpyAsync(o.idx_d.p, o.idx.data(), sizeof(int32_t) * o.idx.size(), cudaMemcpyHostToDevice, s));
    if (o.algo != RF_ALGO_OS && o.algo != RF_ALGO_OS_BINS) {
      // the direct or tensor-core form on the bucket's own kernel set, prepared now so that a
      // reconstruction call launches without synchronising
      o.sub = make_subset(kern, o.idx, s);
      if (o.algo == RF_ALGO_GEMM && o.sub->k) {
        o.sub->gemm_pref_nj = o.gemm_nj;
        o.sub->gemm_pref_s = o.gemm_s;
        gemm_prepare(c, o.sub.get(), o.prec, s);
      }
      continue;
    }
    // partition rows (kernel, partition) of this bucket, contiguous in os_spec
    std::vector<int> gj, gp;
    for (const int j : o.idx)
      for (int p = 0; p < parts[j]; ++p) {
        gj.push_back(j);
        gp.push_back(p);
      }
    const int G = (int)gj.size();
    if (!G) continue;
    const int B = o.B, Lp = o.Lp;
    DevBuf gjd, gpd, rows;
    gjd.ensure(sizeof(int) * G);
    gpd.ensure(sizeof(int) * G);
    RF_CUDA(cudaMemcpyAsync(gjd.p, gj.data(), sizeof(int) * G, cudaMemcpyHostToDevice, s));
    RF_CUDA(cudaMemcpyAsync(gpd.p, gp.data(), sizeof(int) * G, cudaMemcpyHostToDevice, s));
    float2* dst = kern->os_spec.as<float2>() + off[o.idx[0]];
    // FP64 transforms of the partitions, a bounded number of rows at a time
    const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(4096, ((int64_t)256 << 20) / (3LL * B * 16)));
    rows.ensure((size_t)3 * chunk * B * sizeof(double2));
    double2* in = rows.as<double2>();
    double2* out = in + (int64_t)chunk * B;
    double2* tmp = out + (int64_t)chunk * B;
    for (int g0 = 0; g0 < G; g0 += chunk) {
      const int cnt = std::min(chunk, G - g0);
      dim3 grid((unsigned)((B + 255) / 256), (unsigned)cnt);
      k_os_fill<<<grid, 256, 0, s>>>(kern->taps.p, kern->real ? 1 : 0, kern->off_d.as<int64_t>(),
                                     kern->len_d.as<int>(), gjd.as<int>() + g0, gpd.as<int>() + g0, B, Lp, in);
      RF_LAUNCHED();
      fft_c2c_f64(in, out, tmp, B, cnt, -1, c->tw64.as<double2>(), c->n, s);
      const int64_t count = (int64_t)cnt * B;
      if (kern->real) {
        const int64_t hc = (int64_t)cnt * os_row(B, true);
        k_os_round_half<<<(unsigned)((hc + 255) / 256), 256, 0, s>>>(out, cnt, B, 1.0 / (double)B,
                                                                       dst + (int64_t)g0 * os_row(B, true));
      } else if (B == kB2)
        k_os2_round<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(out, count, 1.0 / (double)B,
                                                                     dst + (int64_t)g0 * B);
      else
        k_os_round<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(out, count, 1.0 / (double)B,
                                                                    dst + (int64_t)g0 * B);
      RF_LAUNCHED();
    }
    RF_CUDA(cudaStreamSynchronize(s));  // the row buffers are released at the end of the iteration
  }
  // two-phase buckets: their plan for single-reference calls (the segment spectra come with
  // the call) and its items on the device
  for (int b = 0; b < nb; ++b) {
    OsBucket& o = bk[b];
    if (o.algo != RF_ALGO_OS_BINS || o.idx.empty()) continue;
    std::vector<OsItem> items;
    for (const int j : o.idx)
      items.push_back(OsItem{kern->os_spec.as<float2>() + off[j], nullptr, parts[j], kern->lag0[j], (long long)j});
    o.bins = std::make_shared<BinsPlan>(bins_plan(items, o.B, o.Lp, kern->real, c->n));
    o.bins_items_d.ensure(sizeof(OsItem) * o.bins->items.size());
    RF_CUDA(cudaMemcpy(o.bins_items_d.p, o.bins->items.data(), sizeof(OsItem) * o.bins->items.size(),
                       cudaMemcpyHostToDevice));
    c->bins_y.ensure(o.bins->y_bytes);
    bins_prepare_scratch(c, o.B);
  }
  RF_CUDA(cudaStreamSynchronize(s));
  kern->os_parts = parts;
  kern->os_off = off;
  kern->os_buckets = std::move(bk);
  kern->os_B = kern->os_buckets[0].B;
  kern->os_Lp = kern->os_buckets[0].Lp;
  kern->os_ready = true;
  static unsigned long long version = 0;
  kern->os_version = ++version;
}

void os_prepare(rf_ctx* c, rf_kernels* kern, int B, int Lp, cudaStream_t s) {
  RF_REQUIRE(kern->dtype == RF_F32, "overlap-save needs the FP32 grid");
  RF_REQUIRE(B == 0 || (B >= 512 && B <= kB2 && (B & (B - 1)) == 0 && B <= c->n),
             "overlap-save block %d invalid for n=%lld", B, (long long)c->n);
  if (!B || !Lp) {
    RF_REQUIRE(Lp == 0, "a partition length needs a block size");
    os_choose_layout(c, kern->len, B, kern->real, &B, &Lp);
  }
  const int32_t cut = 0;
  os_prepare_buckets(c, kern, 1, &cut, &B, &Lp, s);
}

// Segment spectra (Q n complex64 for partition ratio Q = B / Lp) plus packed window keys.
size_t os_workspace_bytes(const rf_ctx* c, int32_t k, int64_t W, int Q) {
  const int64_t nw = W > 0 ? (c->n + W - 1) / W : 0;
  return sizeof(float2) * (size_t)Q * (size_t)c->n + sizeof(unsigned long long) * (size_t)k * (size_t)nw + 256;
}

void reconstruct_os(rf_ctx* c, const void* z_ref, rf_kernels* kern, void* z_out, int64_t W, float* max_out,
                    int32_t* argmax_out, cudaStream_t s) {
  if (kern->k == 0) return;
  if (!kern->os_ready) os_prepare(c, kern, 0, 0, s);
  int Qmax = 2;
  for (const OsBucket& bk : kern->os_buckets)
    if (bk.algo == RF_ALGO_OS || bk.algo == RF_ALGO_OS_BINS) Qmax = std::max(Qmax, bk.B / bk.Lp);
  const bool win = max_out != nullptr;
  const size_t need = os_workspace_bytes(c, kern->k, win ? W : 0, Qmax);
  c->scratch.ensure(need);
  float2* Zs = c->scratch.as<float2>();
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(Zs + (int64_t)Qmax * c->n);
  const int64_t nw = win ? (c->n + W - 1) / W : 0;
  if (win) RF_CUDA(cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * (size_t)kern->k * nw, s));
  // one segment transform and one launch per layout bucket (stream order keeps Zs consistent)
  for (const OsBucket& bk : kern->os_buckets) {
    if (bk.idx.empty()) continue;
    if (bk.algo == RF_ALGO_OS_BINS) {
      // the bucket's segment spectra, then the two-phase launches of its plan
      if (bk.B == kB2)
        launch_os2_segments(c, static_cast<const float2*>(z_ref), nullptr, 1, bk.Lp, Zs, s);
      else
        dispatch_bq(bk.B, bk.B / bk.Lp, [&](auto bc, auto qc) {
          constexpr int BB = decltype(bc)::value;
          launch_os_segments<BB>(c, static_cast<const float2*>(z_ref), bk.Lp, Zs, s);
        });
      c->bins_y.ensure(bk.bins->y_bytes);
      bins_prepare_scratch(c, bk.B);
      bins_run(c, *bk.bins, bk.bins_items_d.as<OsItem>(), Zs, c->bins_y.as<float2>(),
               win ? nullptr : static_cast<float2*>(z_out), win ? keys : nullptr, W, s);
      continue;
    }
    if (bk.algo != RF_ALGO_OS) continue;
    if (bk.B == kB2) {
      launch_os2_segments(c, static_cast<const float2*>(z_ref), nullptr, 1, bk.Lp, Zs, s);
      const bool q2 = bk.B / bk.Lp == 2;
      if (win) {
        if (q2) launch_os2<2, true>(c, kern, bk, Zs, nullptr, keys, W, s);
        else launch_os2<4, true>(c, kern, bk, Zs, nullptr, keys, W, s);
      } else {
        if (q2) launch_os2<2, false>(c, kern, bk, Zs, static_cast<float2*>(z_out), nullptr, 0, s);
        else launch_os2<4, false>(c, kern, bk, Zs, static_cast<float2*>(z_out), nullptr, 0, s);
      }
      continue;
    }
    dispatch_bq(bk.B, bk.B / bk.Lp, [&](auto bc, auto qc) {
      constexpr int BB = decltype(bc)::value, QQ = decltype(qc)::value;
      launch_os_segments<BB>(c, static_cast<const float2*>(z_ref), bk.Lp, Zs, s);
      if (win)
        launch_os<BB, QQ, true>(c, kern, bk, Zs, nullptr, keys, W, s);
      else
        launch_os<BB, QQ, false>(c, kern, bk, Zs, static_cast<float2*>(z_out), nullptr, 0, s);
    });
  }
  if (win) {
    const int64_t count = (int64_t)kern->k * nw;
    k_unpack_keys<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(keys, count, max_out, argmax_out);
    RF_LAUNCHED();
  }
  // buckets of the direct or tensor-core form overwrite their rows (after the unpack)
  for (const OsBucket& bk : kern->os_buckets)
    if (bk.algo != RF_ALGO_OS && bk.algo != RF_ALGO_OS_BINS && !bk.idx.empty())
      run_bucket_form(c, z_ref, bk, W, max_out, argmax_out, z_out, 0, s);
}

void reconstruct_batched(rf_ctx* c, int32_t G, const void* const* z_refs, rf_kernels* const* ks, int64_t W,
                         float* max_out, int32_t* argmax_out, cudaStream_t s) {
  // one bucket configuration for the whole batch: the first prepared kernel set decides,
  // else the modelled single layout over all kernel lengths
  const rf_kernels* lead = nullptr;
  for (int g = 0; g < G && !lead; ++g)
    if (ks[g]->os_ready) lead = ks[g];
  std::vector<int32_t> cuts, Bs, Lps;
  std::vector<BucketSpec> spec;
  if (lead) {
    for (const OsBucket& b : lead->os_buckets) {
      cuts.push_back(b.cut_lo);
      Bs.push_back(b.B);
      Lps.push_back(b.Lp);
      const bool os_like = b.algo == RF_ALGO_OS || b.algo == RF_ALGO_OS_BINS;
      spec.push_back(BucketSpec{b.cut_lo, b.algo, b.prec, os_like ? b.B : b.gemm_nj, os_like ? b.Lp : b.gemm_s});
    }
  } else {
    std::vector<int> all;
    for (int g = 0; g < G; ++g) all.insert(all.end(), ks[g]->len.begin(), ks[g]->len.end());
    int B = 0, Lp = 0;
    os_choose_layout(c, all, 0, ks[0]->real, &B, &Lp);
    cuts.push_back(0);
    Bs.push_back(B);
    Lps.push_back(Lp);
    spec.push_back(BucketSpec{0, RF_ALGO_OS, RF_PREC_NATIVE, B, Lp});
  }
  const int nb = (int)cuts.size();
  for (int g = 1; g < G; ++g)
    RF_REQUIRE(ks[g]->real == ks[0]->real, "the kernel sets of a batch are all complex or all real-form");
  const int herm = ks[0]->real ? 1 : 0;
  for (int g = 0; g < G; ++g) os_prepare_forms(c, ks[g], nb, spec.data(), s);
  const int64_t n = c->n;
  const int64_t nw = (n + W - 1) / W;
  // plan key: window, references and kernel sets with their spectra versions (which change
  // whenever a layout changes)
  std::vector<unsigned long long> key;
  key.push_back((unsigned long long)W);
  for (int g = 0; g < G; ++g) {
    key.push_back((unsigned long long)(uintptr_t)z_refs[g]);
    key.push_back((unsigned long long)(uintptr_t)ks[g]);
    key.push_back(ks[g]->os_version);
  }
  int64_t rows = 0;
  for (int g = 0; g < G; ++g) rows += ks[g]->k;
  size_t zs_need = 16;
  for (int b = 0; b < nb; ++b)
    if (spec[b].algo == RF_ALGO_OS || spec[b].algo == RF_ALGO_OS_BINS)
      zs_need = std::max(zs_need, sizeof(float2) * (size_t)G * (size_t)(n / Lps[b]) * Bs[b]);
  if (key != c->batch_key) {
    // work items bucket after bucket (the reference's segment spectra of that bucket's layout)
    std::vector<OsItem> items;
    items.reserve((size_t)rows);
    c->batch_zs.ensure(zs_need);
    const float2* zs_all = c->batch_zs.as<float2>();
    c->batch_lay_off.assign(nb + 1, 0);
    c->batch_unit_off.assign(nb + 1, 0);
    c->batch_sc.assign(nb, 1);
    std::vector<long long> order;
    c->batch_bins.assign(nb, nullptr);
    c->batch_bins_off.assign(nb + 1, 0);
    std::vector<OsItem> bins_all;
    for (int b = 0; b < nb; ++b) {
      if (spec[b].algo == RF_ALGO_OS_BINS) {
        // two-phase bucket: its items (every reference's neighbours in the bucket) and plan
        const int64_t zstride = (n / Lps[b]) * Bs[b];
        std::vector<OsItem> bi;
        int64_t row0 = 0;
        for (int g = 0; g < G; ++g) {
          const rf_kernels* k = ks[g];
          for (const int j : k->os_buckets[b].idx)
            bi.push_back(OsItem{k->os_spec.as<float2>() + k->os_off[j], zs_all + (int64_t)g * zstride,
                                k->os_parts[j], k->lag0[j], (long long)(row0 + j)});
          row0 += k->k;
        }
        c->batch_bins[b] = std::make_shared<BinsPlan>(bins_plan(bi, Bs[b], Lps[b], ks[0]->real, n));
        c->batch_bins_off[b] = (int64_t)bins_all.size();
        bins_all.insert(bins_all.end(), c->batch_bins[b]->items.begin(), c->batch_bins[b]->items.end());
        c->bins_y.ensure(c->batch_bins[b]->y_bytes);
        bins_prepare_scratch(c, Bs[b]);
      }
      if (spec[b].algo != RF_ALGO_OS) {  // direct, tensor-core or two-phase bucket: no work units
        c->batch_lay_off[b + 1] = (int64_t)items.size();
        c->batch_unit_off[b + 1] = (int64_t)order.size();
        continue;
      }
      const int64_t zstride = (n / Lps[b]) * Bs[b];
      const int64_t first = (int64_t)items.size();
      std::vector<int64_t> grp(G + 1, 0);  // items of reference g in this bucket: [grp[g], grp[g+1]) from first
      std::vector<int> pmax(G, 1);
      int64_t row0 = 0;
      for (int g = 0; g < G; ++g) {
        const rf_kernels* k = ks[g];
        for (const int j : k->os_buckets[b].idx) {
          items.push_back(OsItem{k->os_spec.as<float2>() + k->os_off[j], zs_all + (int64_t)g * zstride,
                                 k->os_parts[j], k->lag0[j], (long long)(row0 + j)});
          pmax[g] = std::max(pmax[g], k->os_parts[j]);
        }
        row0 += k->k;
        grp[g + 1] = (int64_t)items.size() - first;
      }
      c->batch_lay_off[b + 1] = (int64_t)items.size();
      const int64_t cnt = grp[G];
      const int B = Bs[b], Lp = Lps[b];
      const int64_t NB = (n + (B - Lp) - 1) / (B - Lp);
      // output blocks per unit: 8, fewer when the units would not fill the GPU a few times
      int SC = 8;
      const int64_t fill = (B == kB2 ? 4LL : 8LL) * c->nsm;
      while (SC > 1 && cnt * ((NB + SC - 1) / SC) < fill) SC /= 2;
      c->batch_sc[b] = SC;
      const int64_t nchunk = (NB + SC - 1) / SC;
      // tiles: a time tile of Ts chunks reads (Ts SC (Q - 1) + P) segment spectra of B values;
      // keep that near 24 MB, and give a tile about as many units as blocks run at once
      const int64_t seg_bytes = (int64_t)B * (int64_t)sizeof(float2);
      const int64_t inflight = B > 16384 ? c->nsm / 2 : (int64_t)c->nsm * (16384 / B);
      for (int g = 0; g < G; ++g) {
        const int64_t lo = first + grp[g], hi = first + grp[g + 1];
        if (lo == hi) continue;
        const int64_t segs = std::max<int64_t>(1, ((int64_t)24 << 20) / seg_bytes - pmax[g]);
        const int64_t Ts = std::max<int64_t>(1, std::min<int64_t>(nchunk, segs / ((int64_t)SC * (B / Lp - 1))));
        const int64_t Tj = std::max<int64_t>(1, std::min<int64_t>(hi - lo, (inflight + Ts - 1) / Ts));
        for (int64_t c0 = 0; c0 < nchunk; c0 += Ts)
          for (int64_t j0 = lo; j0 < hi; j0 += Tj)
            for (int64_t it = j0; it < std::min(hi, j0 + Tj); ++it)
              for (int64_t ch = c0; ch < std::min(nchunk, c0 + Ts); ++ch)
                order.push_back((long long)((it - first) * nchunk + ch));
      }
      c->batch_unit_off[b + 1] = (int64_t)order.size();
    }
    std::vector<const float2*> zp(G);
    for (int g = 0; g < G; ++g) zp[g] = static_cast<const float2*>(z_refs[g]);
    c->batch_key.clear();
    c->batch_items.ensure(std::max<size_t>(16, sizeof(OsItem) * items.size()));
    c->batch_zptr.ensure(sizeof(const float2*) * G);
    c->batch_keys.ensure(sizeof(unsigned long long) * ((size_t)rows * nw + nb));
    if (!items.empty())
      RF_CUDA(cudaMemcpy(c->batch_items.p, items.data(), sizeof(OsItem) * items.size(), cudaMemcpyHostToDevice));
    c->batch_bins_items.ensure(std::max<size_t>(16, sizeof(OsItem) * bins_all.size()));
    if (!bins_all.empty())
      RF_CUDA(cudaMemcpy(c->batch_bins_items.p, bins_all.data(), sizeof(OsItem) * bins_all.size(),
                         cudaMemcpyHostToDevice));
    c->batch_order.ensure(std::max<size_t>(16, sizeof(long long) * order.size()));
    if (!order.empty())
      RF_CUDA(cudaMemcpy(c->batch_order.p, order.data(), sizeof(long long) * order.size(), cudaMemcpyHostToDevice));
    RF_CUDA(cudaMemcpy(c->batch_zptr.p, zp.data(), sizeof(const float2*) * G, cudaMemcpyHostToDevice));
    c->batch_key = key;
    c->batch_rows = rows;
    c->batch_nw = nw;
  }
  if (!rows) return;
  unsigned long long* keys = c->batch_keys.as<unsigned long long>();
  RF_CUDA(cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * ((size_t)rows * nw + nb), s));
  RF_REQUIRE(G <= 65535, "at most 65535 references per batch");
  for (int b = 0; b < nb; ++b) {
    if (spec[b].algo == RF_ALGO_OS_BINS) {
      const BinsPlan& pl = *c->batch_bins[b];
      if (pl.items.empty()) continue;
      if (Bs[b] == kB2)
        launch_os2_segments(c, nullptr, c->batch_zptr.as<const float2*>(), G, Lps[b], c->batch_zs.as<float2>(), s);
      else
        dispatch_bq(Bs[b], Bs[b] / Lps[b], [&](auto bc, auto qc) {
          constexpr int BB = decltype(bc)::value;
          const float2* tw = c->twb32.as<float2>() + c->twb_off[BlockFFTShape<BB>::LOGB];
          auto seg = k_os_segments_batched<BB>;
          RF_CUDA(cudaFuncSetAttribute(seg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)os_smem<BB>()));
          seg<<<dim3((unsigned)(n / Lps[b]), (unsigned)G), BB / 16, os_smem<BB>(), s>>>(
              c->batch_zptr.as<const float2*>(), n, Lps[b], tw, c->batch_zs.as<float2>());
          RF_LAUNCHED();
        });
      bins_run(c, pl, c->batch_bins_items.as<OsItem>() + c->batch_bins_off[b], nullptr, c->bins_y.as<float2>(),
               nullptr, keys, W, s);
      continue;
    }
    const int64_t first = c->batch_lay_off[b], cnt = c->batch_lay_off[b + 1] - first;
    if (!cnt) continue;
    const int B = Bs[b], Lp = Lps[b];
    const int NQ = (int)(n / Lp);
    const int NB = (int)((n + (B - Lp) - 1) / (B - Lp));
    const int SC = c->batch_sc[b];
    const int nchunk = (NB + SC - 1) / SC;
    if (B == kB2) {
      // CTA pairs: one cluster per (chunk of output blocks, work item), no work counter
      launch_os2_segments(c, nullptr, c->batch_zptr.as<const float2*>(), G, Lp, c->batch_zs.as<float2>(), s);
      const float2* tw = c->twb32.as<float2>() + c->twb_off[14];
      const float2* twc = c->twb32.as<float2>() + c->twb_off[15];
      const int fastwin = (W >= 256) ? 1 : 0;
      auto run = [&](auto fn) {
        RF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)os2_smem()));
        for (int64_t done = 0; done < cnt; done += 65535) {
          const int part = (int)std::min<int64_t>(65535, cnt - done);
          fn<<<dim3((unsigned)(2 * nchunk), (unsigned)part), kBH / 16, os2_smem(), s>>>(
              c->batch_items.as<OsItem>() + first + done, nchunk, tw, twc, n, NQ, NB, SC, keys, W, nw, fastwin);
          RF_LAUNCHED();
        }
      };
      if (B / Lp == 2) run(k_os2_batched<2>);
      else run(k_os2_batched<4>);
      continue;
    }
    const int64_t units = c->batch_unit_off[b + 1] - c->batch_unit_off[b];
    RF_REQUIRE(units == cnt * nchunk, "batched plan: unit count");
    unsigned long long* counter = keys + rows * nw + b;
    dispatch_bq(B, B / Lp, [&](auto bc, auto qc) {
      constexpr int BB = decltype(bc)::value, QQ = decltype(qc)::value;
      const int fastwin = (W >= os_warp_span<BB, QQ>()) ? 1 : 0;  // a warp's outputs span <= 2 windows
      const float2* tw = c->twb32.as<float2>() + c->twb_off[BlockFFTShape<BB>::LOGB];
      auto seg = k_os_segments_batched<BB>;
      RF_CUDA(cudaFuncSetAttribute(seg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)os_smem<BB>()));
      seg<<<dim3((unsigned)NQ, (unsigned)G), BB / 16, os_smem<BB>(), s>>>(c->batch_zptr.as<const float2*>(), n, Lp,
                                                                         tw, c->batch_zs.as<float2>());
      RF_LAUNCHED();
      auto fn = k_os_batched<BB, QQ>;
      RF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)os_smem<BB>()));
      int per_sm = 0;
      RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, BB / 16, os_smem<BB>()));
      const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * c->nsm, units));
      fn<<<(unsigned)grid, BB / 16, os_smem<BB>(), s>>>(c->batch_items.as<OsItem>() + first,
                                                        c->batch_order.as<long long>() + c->batch_unit_off[b], units,
                                                        nchunk, tw, n, NQ, NB, SC, keys, W, nw, fastwin, herm,
                                                        counter);
      RF_LAUNCHED();
    });
  }
  const int64_t count = rows * nw;
  k_unpack_keys<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(keys, count, max_out, argmax_out);
  RF_LAUNCHED();
  // buckets of the direct or tensor-core form, group by group, into their rows
  for (int b = 0; b < nb; ++b) {
    if (spec[b].algo == RF_ALGO_OS || spec[b].algo == RF_ALGO_OS_BINS) continue;
    int64_t row0 = 0;
    for (int g = 0; g < G; ++g) {
      const OsBucket& bk = ks[g]->os_buckets[b];
      if (!bk.idx.empty()) run_bucket_form(c, z_refs[g], bk, W, max_out, argmax_out, nullptr, row0, s);
      row0 += ks[g]->k;
    }
  }
}

}  // namespace rf
