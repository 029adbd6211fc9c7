// Two-phase overlap-save for long kernels: the partition sums of Eq. 7's block form computed
// per bin over a run of output blocks, then the block transforms.
//
// Single-pass overlap-save (reconstruct_os.cu) forms, for each output block s of a neighbour,
//   Y_s[k] = sum_{p < P} Zs[(s (Q - 1) - 1 - p) mod NQ][k] C[p][k]
// in the block's own thread block, reading P segment spectra and P partition spectra (32 P
// bytes per output at Q = 2) from L2: long kernels make that L2-bandwidth bound.  Here the
// same sums run with the roles of bins and blocks swapped.  Phase 1: a thread owns one bin k of
// one neighbour, keeps C[p][k] for every p and the last P segment values Zs[.][k] in registers,
// and walks the output blocks s0 .. s0 + ns - 1, one FIR step per block: one 8-byte load of the
// next segment value, 8 P flops, one 8-byte store of Y_s[k] into a buffer.  Moving to block
// s + 1 shifts the window by Q - 1 segments.  Phase 2: one thread block per (neighbour, s)
// reads Y_s and runs the block tail of the single-pass form (inverse transform, series or fused
// window peaks); for 32768-point blocks, a persistent CTA runs the two 16384-point half
// transforms of a block in turn (os_tail.cuh).  Same arithmetic per output (the products in the
// same FP32 operations, summed in another order), so the error bound is that of the single-pass
// form.
//
// Waves: the neighbours of a bucket, sorted by partition count, are cut into tiles of T items;
// each tile runs every output block in time tiles of ns blocks, phase 1 then phase 2 per
// (item tile, time tile).  Waves alternate two buffers, phase 1 on the caller's stream and
// phase 2 on a second stream (events order them; no kernel waits on another).  Kernels with
// more than kBinsPMax = 40 partitions take several phase-1 passes, each adding its partitions to
// the buffer.
#include <algorithm>
#include <type_traits>
#include <utility>
#include <vector>

#include "os_tail.cuh"
#include "rf_internal.h"

namespace rf {

namespace {

constexpr int kBinsThreads = 128;
// Blocks per SM that phase 1 asks the register allocator for: the window of PM partitions takes
// four registers per partition in the ring and the partition values, so fewer partitions leave
// room for more warps.
template <int PM>
__host__ __device__ constexpr int bins_min_blocks() {
  return PM <= 16 ? 4 : (PM <= 24 ? 3 : 2);
}
constexpr int kBinsPMax = 40;

// f(std::integral_constant<int, u>) for u = 0 .. N - 1, unrolled at compile time.
template <int N, typename F, int... U>
__device__ __forceinline__ void unroll_steps_impl(F&& f, std::integer_sequence<int, U...>) {
  (f(std::integral_constant<int, U>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void unroll_steps(F&& f) {
  unroll_steps_impl<N>(f, std::make_integer_sequence<int, N>{});
}

// Phase 1.  Block (bin slice, item): thread k = slice * 128 + tid.  Partitions p0 .. p0 + PM - 1
// of each item (those below its P); `accumulate` adds to the buffer (passes after the first).
// Zs: per-item segment spectra, or zs_one for every item when not null.  Y: [item][ns][B].
template <int PM, int Q>
__global__ void __launch_bounds__(kBinsThreads, bins_min_blocks<PM>())
    k_bins_products(const OsItem* __restrict__ items, const float2* __restrict__ zs_one, int B, int NQ, int crow,
                    int herm, int s0, int ns, int p0, int accumulate, float2* __restrict__ Y) {
  const int ii = blockIdx.y;
  const OsItem it = items[ii];
  const int k = blockIdx.x * kBinsThreads + threadIdx.x;
  const float2* Zs = zs_one ? zs_one : it.Zs;
  const int pc = min(PM, it.P - p0);  // partitions of this pass (may be <= 0: nothing to add)
  float2* y = Y + (int64_t)ii * ns * B + k;
  if (pc <= 0) {
    if (!accumulate)
      for (int si = 0; si < ns; ++si) y[(int64_t)si * B] = make_float2(0.f, 0.f);
    return;
  }
  // partition values of this bin; a real-form set stores bins 0..B/2, the others are mirrors
  const bool mir = herm && k > B / 2;
  const int kk = mir ? B - k : k;
  const float cs = mir ? -1.f : 1.f;
  float2 c[PM];
#pragma unroll
  for (int p = 0; p < PM; ++p) {
    float2 v = make_float2(0.f, 0.f);
    if (p < pc) {
      v = __ldg(it.C + (int64_t)(p0 + p) * crow + kk);
      v.y *= cs;
    }
    c[p] = v;
  }
  // window of block s0: w[p] = Zs[(s0 (Q - 1) - 1 - p0 - p) mod NQ][k] (NQ a power of two)
  const int qmask = NQ - 1;
  float2 w[PM];
#pragma unroll
  for (int p = 0; p < PM; ++p)
    w[p] = p < pc ? __ldcg(Zs + (int64_t)((s0 * (Q - 1) - 1 - p0 - p) & qmask) * B + k) : make_float2(0.f, 0.f);
  // The window as a ring of registers inside a group of U steps: at step u, logical entry p sits
  // in register (p - (Q - 1) u) mod PM, so moving to the next block renames registers (the Q - 1
  // newest values take the oldest ones' registers) instead of moving values; after the group one
  // rotation by (Q - 1) U restores entry p to register p.  U = 8 keeps the unrolled code small
  // enough for the instruction cache and the rotation at 2 PM / U moves per step.
  //
  // The entering values come through a second ring of DP register slots (DP divides U): at the
  // start of a group, slot d holds the values entering at block s0 + si + 1 + d; step u takes
  // slot u mod DP and refills it with the values of DP blocks later, so that every load has DP
  // steps of multiply-adds to arrive.  A last partial group loads its values directly.
  constexpr int U = 8;
  constexpr int DP = Q == 2 ? 8 : 2;
  static_assert(U % DP == 0, "prefetch ring");
  auto seg_load = [&](int sb, int p) {
    return __ldcg(Zs + (int64_t)((sb * (Q - 1) - 1 - p0 - p) & qmask) * B + k);
  };
  float2 pf[DP][Q - 1];
#pragma unroll
  for (int d = 0; d < DP; ++d)
#pragma unroll
    for (int p = 0; p < Q - 1; ++p) pf[d][p] = seg_load(s0 + 1 + d, p);
  auto step = [&](int si, auto uc, auto rc) {
    constexpr int u = decltype(uc)::value;
    constexpr bool ring = decltype(rc)::value;
    float2 nn[Q - 1];
#pragma unroll
    for (int p = 0; p < Q - 1; ++p) nn[p] = seg_load(ring ? s0 + si + 1 + DP : s0 + si + 1, p);
    float2 a[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) a[r] = make_float2(0.f, 0.f);
#pragma unroll
    for (int p = 0; p < PM; ++p) {
      const float2 wv = w[((p - (Q - 1) * u) % PM + PM) % PM];
      float2& acc = a[p & 3];
      acc.x = fmaf(wv.x, c[p].x, fmaf(-wv.y, c[p].y, acc.x));
      acc.y = fmaf(wv.x, c[p].y, fmaf(wv.y, c[p].x, acc.y));
    }
    float2 sum = make_float2((a[0].x + a[1].x) + (a[2].x + a[3].x), (a[0].y + a[1].y) + (a[2].y + a[3].y));
    float2* yp = y + (int64_t)si * B;
    if (accumulate) {
      const float2 prev = *yp;
      sum.x += prev.x;
      sum.y += prev.y;
    }
    *yp = sum;
#pragma unroll
    for (int p = 0; p < Q - 1; ++p) {
      float2& r = w[((p - (Q - 1) * (u + 1)) % PM + PM) % PM];
      if constexpr (ring) {
        r = pf[u % DP][p];
        pf[u % DP][p] = nn[p];
      } else {
        r = nn[p];
      }
    }
  };
  // entry p back in register p after a group of G steps
  auto rotate = [&](auto gc) {
    constexpr int G = decltype(gc)::value;
    float2 t[PM];
#pragma unroll
    for (int p = 0; p < PM; ++p) t[p] = w[((p - (Q - 1) * G) % PM + PM) % PM];
#pragma unroll
    for (int p = 0; p < PM; ++p) w[p] = t[p];
  };
  int si = 0;
  for (; si + U <= ns; si += U) {
    unroll_steps<U>([&](auto uc) { step(si + decltype(uc)::value, uc, std::true_type{}); });
    rotate(std::integral_constant<int, U>{});
  }
  for (; si < ns; ++si) {
    step(si, std::integral_constant<int, 0>{}, std::false_type{});
    rotate(std::integral_constant<int, 1>{});
  }
}

// Phase 2.  Block (s - s0, item): the partition sums of block s from the buffer, then the block
// tail: series rows z_out + row n, or window keys rows keys + row nw.
template <int B, int Q, bool WINMAX>
__global__ void __launch_bounds__(B / 16, 16384 / B)
    k_bins_tail(const OsItem* __restrict__ items, const float2* __restrict__ Y, int s0, int ns,
                const float2* __restrict__ tw, int64_t n, float2* __restrict__ z_out,
                unsigned long long* __restrict__ keys, int64_t W, int64_t nw, int fastwin) {
  extern __shared__ float2 sm[];
  const int si = blockIdx.x, ii = blockIdx.y;
  const OsItem it = items[ii];
  const float2* y = Y + ((int64_t)ii * ns + si) * B + threadIdx.x;
  float2 v[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) v[t] = __ldcg(y + t * (B / 16));
  os_block_tail<B, Q, WINMAX>(v, s0 + si, it.lag0, n, WINMAX ? nullptr : z_out + it.row * n,
                              WINMAX ? keys + it.row * nw : nullptr, W, nw, fastwin, tw, sm);
}

// Phase 2 of the 32768-point layout (Q = 2) on one CTA per block (os_tail.cuh: both half
// transforms in turn, no cluster exchange).  Persistent: CTA b takes the units
// u = b, b + gridDim.x, .. of the wave's (item, block) units, with scratch row b.
template <bool WINMAX>
__global__ void __launch_bounds__(kBH / 16, 1)
    k_bins_tail_pair(const OsItem* __restrict__ items, const float2* __restrict__ Y, int s0, int ns, int units,
                     const float2* __restrict__ tw, const float2* __restrict__ twc, int64_t n,
                     float2* __restrict__ z_out, unsigned long long* __restrict__ keys, int64_t W, int64_t nw,
                     int fastwin, float2* __restrict__ e0_all) {
  extern __shared__ float2 sm[];
  constexpr int NT = kBH / 16;
  const int tid = threadIdx.x;
  float2* e0 = e0_all + (int64_t)blockIdx.x * kBH;
  for (int u = blockIdx.x; u < units; u += gridDim.x) {
    const int ii = u / ns, si = u - ii * ns;
    const float2* y = Y + ((int64_t)u) * kB2 + tid;  // unit u = (item ii, block si) of the wave
    pair1_halves(
        [&](int h, float2(&v)[16]) {
#pragma unroll
          for (int t = 0; t < 16; ++t) v[t] = __ldcg(y + h * kBH + t * NT);
        },
        e0, tw, sm);
    const int64_t lag0 = items[ii].lag0, row = items[ii].row;  // read after the transforms
    pair1_tail<WINMAX>(e0, twc, s0 + si, lag0, n, WINMAX ? nullptr : z_out + row * n,
                       WINMAX ? keys + row * nw : nullptr, W, nw, fastwin, sm);
  }
}

template <int PM, int Q>
void launch_products(const OsItem* items, const float2* zs_one, int B, int NQ, int crow, int herm, int s0, int ns,
                     int p0, int accumulate, float2* Y, int nitems, cudaStream_t s) {
  dim3 grid((unsigned)(B / kBinsThreads), (unsigned)nitems);
  k_bins_products<PM, Q><<<grid, kBinsThreads, 0, s>>>(items, zs_one, B, NQ, crow, herm, s0, ns, p0, accumulate, Y);
  RF_LAUNCHED();
}

// The smallest register window that holds pm partitions: steps of 4 at Q = 2 (the long-kernel
// layouts), of 8 at Q = 4.
template <int Q>
void products_pm(int pm, const OsItem* items, const float2* zs_one, int B, int NQ, int crow, int herm, int s0,
                 int ns, int p0, int accumulate, float2* Y, int nitems, cudaStream_t s) {
#define RF_BINS_PM(PMV)                                                                                          \
  if (pm <= PMV) return launch_products<PMV, Q>(items, zs_one, B, NQ, crow, herm, s0, ns, p0, accumulate, Y, \
                                                nitems, s);
  RF_BINS_PM(8)
  if constexpr (Q == 2) {
    RF_BINS_PM(12)
  }
  RF_BINS_PM(16)
  if constexpr (Q == 2) {
    RF_BINS_PM(20)
  }
  RF_BINS_PM(24)
  if constexpr (Q == 2) {
    RF_BINS_PM(28)
  }
  RF_BINS_PM(32)
  if constexpr (Q == 2) {
    RF_BINS_PM(36)
  }
#undef RF_BINS_PM
  launch_products<kBinsPMax, Q>(items, zs_one, B, NQ, crow, herm, s0, ns, p0, accumulate, Y, nitems, s);
}

template <int B, int Q, bool WINMAX>
void launch_tail(const OsItem* items, const float2* Y, int s0, int ns, int nitems, const float2* tw, int64_t n,
                 float2* z_out, unsigned long long* keys, int64_t W, int64_t nw, int fastwin, cudaStream_t s) {
  const size_t smem = sizeof(float2) * BlockFFTShape<B>::SMEM;
  auto fn = k_bins_tail<B, Q, WINMAX>;
  RF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  fn<<<dim3((unsigned)ns, (unsigned)nitems), B / 16, smem, s>>>(items, Y, s0, ns, tw, n, z_out, keys, W, nw,
                                                                fastwin);
  RF_LAUNCHED();
}

template <bool WINMAX>
void launch_tail_pair(rf_ctx* c, const OsItem* items, const float2* Y, int s0, int ns, int nitems, int64_t n,
                      float2* z_out, unsigned long long* keys, int64_t W, int64_t nw, cudaStream_t s) {
  auto fn = k_bins_tail_pair<WINMAX>;
  const size_t smem = os2_tail_smem();  // the transform's shared memory, then BH magnitudes
  RF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int units = ns * nitems;
  const int grid = std::min(units, c->nsm);
  RF_REQUIRE(c->bins_e0.bytes >= sizeof(float2) * (size_t)kBH * (size_t)grid,
             "two-phase 32768-point tail: scratch not prepared");
  const int fastwin = (WINMAX && W >= pair1_warp_span()) ? 1 : 0;
  const float2* tw = c->twb32.as<float2>() + c->twb_off[14];
  const float2* twc = c->twb32.as<float2>() + c->twb_off[15];
  fn<<<grid, kBH / 16, smem, s>>>(items, Y, s0, ns, units, tw, twc, n, z_out, keys, W, nw, fastwin,
                                  c->bins_e0.as<float2>());
  RF_LAUNCHED();
}

template <bool WINMAX>
void tail_bq(int B, int Q, const OsItem* items, const float2* Y, int s0, int ns, int nitems, const float2* tw,
             int64_t n, float2* z_out, unsigned long long* keys, int64_t W, int64_t nw, int fastwin, cudaStream_t s) {
#define RF_BINS_TAIL(BB, QQ) \
  if (B == BB && Q == QQ) return launch_tail<BB, QQ, WINMAX>(items, Y, s0, ns, nitems, tw, n, z_out, keys, W, nw, fastwin, s);
  RF_BINS_TAIL(4096, 2)
  RF_BINS_TAIL(4096, 4)
  RF_BINS_TAIL(8192, 2)
  RF_BINS_TAIL(8192, 4)
  RF_BINS_TAIL(16384, 2)
  RF_BINS_TAIL(16384, 4)
#undef RF_BINS_TAIL
  RF_REQUIRE(false, "two-phase overlap-save: no block tail for B=%d, Q=%d", B, Q);
}

}  // namespace

void bins_prepare_scratch(rf_ctx* c, int B) {
  if (B == kB2) c->bins_e0.ensure(sizeof(float2) * (size_t)kBH * (size_t)c->nsm);
  if (!c->bins_side) {
    RF_CUDA(cudaStreamCreateWithFlags(&c->bins_side, cudaStreamNonBlocking));
    for (cudaEvent_t& e : c->bins_ev) RF_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
}

bool bins_layout_ok(int B, int Lp) {
  return ((B == 4096 || B == 8192 || B == 16384) && (Lp == B / 2 || Lp == B / 4)) || (B == kB2 && Lp == kBH);
}

BinsPlan bins_plan(std::vector<OsItem> items, int B, int Lp, bool herm, int64_t n) {
  RF_REQUIRE(bins_layout_ok(B, Lp), "two-phase overlap-save takes B in {4096, 8192, 16384} with Lp = B/2 or B/4, "
                                    "or B = 32768 with Lp = 16384");
  RF_REQUIRE(!(herm && B == kB2), "real-form kernels take two-phase blocks of at most 16384 points");
  BinsPlan pl;
  pl.B = B;
  pl.Lp = Lp;
  pl.herm = herm;
  pl.NQ = (int)(n / Lp);
  pl.NB = (int)((n + (B - Lp) - 1) / (B - Lp));
  // most partitions first, so that a tile's register window fits its items closely
  std::stable_sort(items.begin(), items.end(), [](const OsItem& a, const OsItem& b) { return a.P > b.P; });
  pl.items = std::move(items);
  const int cnt = (int)pl.items.size();
  // tiles of T items x ns blocks: a buffer of about 2048 blocks' sums (256 MB at B = 16384)
  const int T = std::max(1, std::min(cnt, 16));
  const int ns = (int)std::max<int64_t>(1, std::min<int64_t>(pl.NB, (2048 + T - 1) / T));
  for (int i0 = 0; i0 < cnt; i0 += T) {
    const int m = std::min(T, cnt - i0);
    int pmax = 1;
    for (int q = i0; q < i0 + m; ++q) pmax = std::max(pmax, pl.items[q].P);
    for (int s0 = 0; s0 < pl.NB; s0 += ns)
      pl.waves.push_back(BinsWave{i0, m, s0, (int)std::min<int64_t>(ns, pl.NB - s0), pmax});
  }
  pl.y_stride = (size_t)T * (size_t)ns * (size_t)B;
  pl.y_bytes = 2 * sizeof(float2) * pl.y_stride + 256;
  return pl;
}

void bins_run(rf_ctx* c, const BinsPlan& pl, const OsItem* items_dev, const float2* zs_one, float2* Y,
              float2* z_out, unsigned long long* keys, int64_t W, cudaStream_t s) {
  const int B = pl.B, Q = B / pl.Lp;
  const int64_t n = c->n;
  const bool win = keys != nullptr;
  const int64_t nw = win ? (n + W - 1) / W : 0;
  int logb = 0;
  while ((1 << logb) < B) ++logb;
  const float2* twb = c->twb32.as<float2>() + c->twb_off[logb];
  const int crow = os_row(B, pl.herm);
  // a warp's outputs in the epilogue span at most two windows when W covers 32 threads' runs
  const int fastwin = (win && W >= 32 * ((B - pl.Lp) / (B / 16))) ? 1 : 0;
  // Phase 1 of every wave on s, phase 2 on the side stream; wave w uses buffer w mod 2, so
  // phase 1 of wave w + 1 may run beside phase 2 of wave w.  Edges: phase 2 of w after phase 1
  // of w; phase 1 of w + 2 (same buffer) after phase 2 of w; the caller's stream after the last
  // phase 2.  Under stream capture the events become the graph's edges (fork and join).
  RF_REQUIRE(c->bins_side != nullptr, "two-phase overlap-save: side stream not prepared");
  RF_REQUIRE(c->bins_y.bytes >= pl.y_bytes, "two-phase overlap-save: buffer not prepared");
  cudaStream_t side = c->bins_side;
  cudaEvent_t* ev = c->bins_ev;  // [0] fork, [1] join, [2 + b] phase 1 done, [4 + b] phase 2 done
  RF_CUDA(cudaEventRecord(ev[0], s));
  RF_CUDA(cudaStreamWaitEvent(side, ev[0], 0));
  for (size_t w = 0; w < pl.waves.size(); ++w) {
    const BinsWave& wv = pl.waves[w];
    const int b = (int)(w & 1);
    float2* Yw = Y + (size_t)b * pl.y_stride;
    const OsItem* it = items_dev + wv.item0;
    if (w >= 2) RF_CUDA(cudaStreamWaitEvent(s, ev[4 + b], 0));
    for (int p0 = 0; p0 < wv.pmax; p0 += kBinsPMax) {
      const int pm = std::min(kBinsPMax, wv.pmax - p0);
      if (Q == 2)
        products_pm<2>(pm, it, zs_one, B, pl.NQ, crow, pl.herm, wv.s0, wv.ns, p0, p0 > 0, Yw, wv.nitems, s);
      else
        products_pm<4>(pm, it, zs_one, B, pl.NQ, crow, pl.herm, wv.s0, wv.ns, p0, p0 > 0, Yw, wv.nitems, s);
    }
    RF_CUDA(cudaEventRecord(ev[2 + b], s));
    RF_CUDA(cudaStreamWaitEvent(side, ev[2 + b], 0));
    if (B == kB2) {
      if (win)
        launch_tail_pair<true>(c, it, Yw, wv.s0, wv.ns, wv.nitems, n, nullptr, keys, W, nw, side);
      else
        launch_tail_pair<false>(c, it, Yw, wv.s0, wv.ns, wv.nitems, n, z_out, nullptr, W, 0, side);
    } else if (win) {
      tail_bq<true>(B, Q, it, Yw, wv.s0, wv.ns, wv.nitems, twb, n, nullptr, keys, W, nw, fastwin, side);
    } else {
      tail_bq<false>(B, Q, it, Yw, wv.s0, wv.ns, wv.nitems, twb, n, z_out, nullptr, W, 0, 0, side);
    }
    RF_CUDA(cudaEventRecord(ev[4 + b], side));
  }
  RF_CUDA(cudaEventRecord(ev[1], side));
  RF_CUDA(cudaStreamWaitEvent(s, ev[1], 0));
}

}  // namespace rf

// the two-phase side stream and events (created by rf::bins_prepare_scratch)
rf_ctx::~rf_ctx() {
  for (cudaEvent_t e : bins_ev)
    if (e) cudaEventDestroy(e);
  if (bins_side) cudaStreamDestroy(bins_side);
}
