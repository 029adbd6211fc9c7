// Direct reconstruction on CUDA cores (Eq. 8, circular discrete form):
//   z_j[i] = sum_{l < L_j} c_j[l] z_ref[(i - m0_j - l) mod n]
// and the fused per-window peak (max |z_j|^2 and its first index).
//
// A block owns a range of outputs of one neighbour and walks it in tiles of
// NT*E samples; taps are consumed in chunks of LC.  Per tap chunk the block
// stages the z_ref strip the tile needs in shared memory (padded one slot per
// E entries so that the per-thread stride of E is bank-conflict free).  Each
// thread owns E consecutive outputs and keeps the E strip values it needs in
// registers, sliding them by one sample per tap: one shared load and one
// broadcast tap load per E complex multiply-adds.  Real-form kernels (real taps T = R) take
// complex x real products: two multiply-adds per tap and output instead of four.
#include <cfloat>
#include <type_traits>

#include "cplx.cuh"
#include "rf_internal.h"

namespace rf {

namespace {

template <typename R>
struct Best {
  R v;
  long long i;
};

template <typename R>
__device__ __forceinline__ bool better(R v, long long i, R bv, long long bi) {
  return v > bv || (v == bv && i < bi);
}

// Block-wide (value, index) maximum with lowest-index ties.  All threads get the result.
template <typename R, int NT>
__device__ Best<R> block_best(R v, long long i) {
  __shared__ R sv[NT / 32];
  __shared__ long long si[NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const R ov = __shfl_down_sync(0xffffffffu, v, o);
    const long long oi = __shfl_down_sync(0xffffffffu, i, o);
    if (better(ov, oi, v, i)) {
      v = ov;
      i = oi;
    }
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sv[w] = v;
    si[w] = i;
  }
  __syncthreads();
  Best<R> b{sv[0], si[0]};
  for (int q = 1; q < NT / 32; ++q)
    if (better(sv[q], si[q], b.v, b.i)) b = Best<R>{sv[q], si[q]};
  __syncthreads();
  return b;
}

template <typename V, typename T, int E, int NT, int LC, bool WINMAX>
__global__ void __launch_bounds__(NT) k_direct(const V* __restrict__ z_ref, int64_t n, const T* __restrict__ taps,
                                               const int64_t* __restrict__ off, const int* __restrict__ len,
                                               const int* __restrict__ lag0, int64_t range, V* __restrict__ z_out,
                                               int64_t W, int64_t nw, float* __restrict__ max_out,
                                               int* __restrict__ arg_out) {
  using R = typename real_of<V>::type;
  constexpr bool REAL = std::is_same<T, R>::value;
  constexpr int TILE = NT * E;
  constexpr int SPAN = TILE + LC;               // strip entries (last one unused)
  constexpr int PAD = SPAN + SPAN / E + 1;       // padded strip size
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* strip = reinterpret_cast<V*>(smem_raw);
  T* tp = reinterpret_cast<T*>(strip + PAD);
  R* mag = reinterpret_cast<R*>(tp + LC);
  Best<R>* run = reinterpret_cast<Best<R>*>(mag + TILE);  // running best per window of the range

  const int j = blockIdx.y;
  const int L = len[j];
  const int64_t m0 = lag0[j];
  const T* c = taps + off[j];
  const int64_t mask = n - 1;
  const int64_t r0 = (int64_t)blockIdx.x * range;
  const int64_t r1 = min(n, r0 + range);
  const int tid = threadIdx.x;
  const int64_t w_first = WINMAX ? r0 / W : 0;
  const int64_t w_last = WINMAX ? (r1 - 1) / W : 0;
  if (WINMAX) {
    for (int64_t w = w_first + tid; w <= w_last; w += NT) run[w - w_first] = Best<R>{(R)-1, 0};
  }

  for (int64_t c0 = r0; c0 < r1; c0 += TILE) {
    V acc[E];
#pragma unroll
    for (int e = 0; e < E; ++e) acc[e] = cmake<V>((R)0, (R)0);
    for (int l0 = 0; l0 < L; l0 += LC) {
      const int lc = min(LC, L - l0);
      __syncthreads();
      // strip[p] = z_ref[(c0 - m0 - l0 - LC + 1 + p) mod n]
      const int64_t base = c0 - m0 - l0 - LC + 1;
      for (int p = tid; p < SPAN - 1; p += NT) strip[p + p / E] = z_ref[(base + p) & mask];
      for (int r = tid; r < LC; r += NT) {
        if constexpr (REAL) tp[r] = (r < lc) ? c[l0 + r] : (R)0;
        else tp[r] = (r < lc) ? c[l0 + r] : cmake<V>((R)0, (R)0);
      }
      __syncthreads();
      const int p0 = tid * E + LC - 1;
      V win[E], part[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        win[e] = strip[(p0 + e) + (p0 + e) / E];
        part[e] = cmake<V>((R)0, (R)0);
      }
#pragma unroll 2
      for (int r = 0; r < LC; ++r) {
        const T cr = tp[r];
#pragma unroll
        for (int e = 0; e < E; ++e) {
          if constexpr (REAL) {
            part[e].x = fma(cr, win[e].x, part[e].x);
            part[e].y = fma(cr, win[e].y, part[e].y);
          } else {
            part[e].x = fma(cr.x, win[e].x, part[e].x);
            part[e].x = fma(-cr.y, win[e].y, part[e].x);
            part[e].y = fma(cr.x, win[e].y, part[e].y);
            part[e].y = fma(cr.y, win[e].x, part[e].y);
          }
        }
#pragma unroll
        for (int e = E - 1; e > 0; --e) win[e] = win[e - 1];
        if (r + 1 < LC) {
          const int q = p0 - r - 1;
          win[0] = strip[q + q / E];
        }
      }
      // two-level summation: per-chunk partial sums keep the FP32 rounding error
      // growth at about sqrt(LC) + sqrt(L / LC) instead of sqrt(L)
#pragma unroll
      for (int e = 0; e < E; ++e) acc[e] = cadd(acc[e], part[e]);
    }
    const int64_t cend = min(r1, c0 + TILE);
    if (!WINMAX) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int64_t i = c0 + tid * E + e;
        if (i < cend) z_out[(int64_t)j * n + i] = acc[e];
      }
    } else {
      __syncthreads();
#pragma unroll
      for (int e = 0; e < E; ++e) mag[tid * E + e] = acc[e].x * acc[e].x + acc[e].y * acc[e].y;
      __syncthreads();
      for (int64_t w = c0 / W; w <= (cend - 1) / W; ++w) {
        const int64_t lo = max(c0, w * W), hi = min(cend, (w + 1) * W);
        R bv = (R)-1;
        long long bi = 0;
        for (int64_t i = lo + tid; i < hi; i += NT) {
          const R v = mag[i - c0];
          if (v > bv) {
            bv = v;
            bi = i;
          }
        }
        const Best<R> b = block_best<R, NT>(bv, bi);
        if (tid == 0) {
          Best<R>& rb = run[w - w_first];
          if (b.v > rb.v) rb = b;  // earlier tiles hold the earlier indices
        }
      }
    }
  }
  if (WINMAX) {
    __syncthreads();
    for (int64_t w = w_first + tid; w <= w_last; w += NT) {
      const Best<R> b = run[w - w_first];
      max_out[(int64_t)j * nw + w] = (float)b.v;
      arg_out[(int64_t)j * nw + w] = (int)b.i;
    }
  }
}

template <typename V, typename T, int E, int NT, int LC, bool WINMAX>
void launch_direct(rf_ctx* c, const rf_kernels* kern, const V* z_ref, V* z_out, int64_t W, float* max_out,
                   int32_t* arg_out, cudaStream_t s) {
  using R = typename real_of<V>::type;
  constexpr int TILE = NT * E;
  constexpr int SPAN = TILE + LC;
  constexpr int PAD = SPAN + SPAN / E + 1;
  const int64_t n = c->n;
  int64_t range, nw = 0, wpc = 0;
  if (WINMAX) {
    nw = (n + W - 1) / W;
    wpc = std::max<int64_t>(1, (TILE + W - 1) / W);  // whole windows per block, at least one tile of work
    range = wpc * W;
  } else {
    range = TILE;
  }
  const int64_t nblk = (n + range - 1) / range;
  const size_t smem = sizeof(V) * PAD + sizeof(T) * LC + sizeof(R) * TILE + sizeof(Best<R>) * (size_t)(wpc + 2) + 16;
  constexpr size_t smem_cap = 200 * 1024;
  RF_REQUIRE(smem <= smem_cap, "direct reconstruct: window of %lld samples needs too much shared memory",
             (long long)W);
  auto kfn = k_direct<V, T, E, NT, LC, WINMAX>;
  // a process-wide attribute of the function: set to the cap that bounds every launch, so that a
  // context on another host thread never lowers it under this launch
  RF_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cap));
  int64_t done = 0;
  while (done < kern->k) {
    const int cnt = (int)std::min<int64_t>(65535, kern->k - done);
    dim3 grid((unsigned)nblk, (unsigned)cnt);
    kfn<<<grid, NT, smem, s>>>(z_ref, n, static_cast<const T*>(kern->taps.p), kern->off_d.as<int64_t>() + done,
                               kern->len_d.as<int>() + done, kern->lag0_d.as<int>() + done, range,
                               z_out ? z_out + done * n : nullptr, W, nw, max_out ? max_out + done * nw : nullptr,
                               arg_out ? arg_out + done * nw : nullptr);
    RF_LAUNCHED();
    done += cnt;
  }
}

// Window peaks of series already in memory: one block per (window, series).
template <typename V, int NT>
__global__ void __launch_bounds__(NT) k_winmax_series(const V* __restrict__ z, int64_t n, int64_t W, int64_t nw,
                                                      float* __restrict__ max_out, int* __restrict__ arg_out) {
  using R = typename real_of<V>::type;
  const int64_t w = blockIdx.x;
  const int64_t row = blockIdx.y;
  const V* zr = z + row * n;
  const int64_t lo = w * W, hi = min(n, (w + 1) * W);
  R bv = (R)-1;
  long long bi = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += NT) {
    const V a = zr[i];
    const R v = a.x * a.x + a.y * a.y;
    if (v > bv) {
      bv = v;
      bi = i;
    }
  }
  const Best<R> b = block_best<R, NT>(bv, bi);
  if (threadIdx.x == 0) {
    max_out[row * nw + w] = (float)b.v;
    arg_out[row * nw + w] = (int)b.i;
  }
}

}  // namespace

void reconstruct_direct(rf_ctx* c, const void* z_ref, const rf_kernels* kern, void* z_out, int64_t W,
                        float* max_out, int32_t* argmax_out, cudaStream_t s) {
  if (kern->k == 0) return;
  const bool win = max_out != nullptr;
  auto run = [&](auto vtag, auto ttag, auto etag) {
    using V = decltype(vtag);
    using T = decltype(ttag);
    constexpr int E = decltype(etag)::value;
    auto zr = static_cast<const V*>(z_ref);
    auto zo = static_cast<V*>(z_out);
    if (win) launch_direct<V, T, E, 256, 256, true>(c, kern, zr, nullptr, W, max_out, argmax_out, s);
    else launch_direct<V, T, E, 256, 256, false>(c, kern, zr, zo, W, nullptr, nullptr, s);
  };
  using E4 = std::integral_constant<int, 4>;
  using E8 = std::integral_constant<int, 8>;
  if (c->g.dtype == RF_F64) {
    if (kern->real) run(double2{}, double{}, E4{});
    else run(double2{}, double2{}, E4{});
  } else {
    if (kern->real) run(float2{}, float{}, E8{});
    else run(float2{}, float2{}, E8{});
  }
}

void winmax_series(rf_ctx* c, const void* z, int32_t count, int64_t W, float* max_out, int32_t* argmax_out,
                   cudaStream_t s) {
  const int64_t n = c->n;
  const int64_t nw = (n + W - 1) / W;
  RF_REQUIRE(nw <= 0x7fffffff && count <= 65535, "winmax: too many windows or series");
  dim3 grid((unsigned)nw, (unsigned)count);
  if (c->g.dtype == RF_F64)
    k_winmax_series<double2, 256><<<grid, 256, 0, s>>>(static_cast<const double2*>(z), n, W, nw, max_out, argmax_out);
  else
    k_winmax_series<float2, 256><<<grid, 256, 0, s>>>(static_cast<const float2*>(z), n, W, nw, max_out, argmax_out);
  RF_LAUNCHED();
}

}  // namespace rf
