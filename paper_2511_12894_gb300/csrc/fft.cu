// Batched Stockham FFT through global memory (radix 16 passes plus one
// radix-2/4/8 pass), FP32 and FP64.  Eq. (1) sign convention: forward passes
// use exp(-2 pi i j k / n), inverse passes exp(+2 pi i j k / n), unnormalised.
//
// Pass p of radix R, with Ns = product of the earlier radices, maps butterfly
// j in [0, n/R) (k = j mod Ns) as
//   a[t]   = in[j + t n/R] * w^(t k),  w = exp(sign 2 pi i / (Ns R)),  t < R
//   a      = DFT_R(a)
//   out[(j - k) R + k + t Ns] = a[t]
// which leaves the transform in natural order after the last pass (Stockham
// autosort).  Consecutive threads take consecutive j, so every load and (for
// Ns >= 32) every store of a warp is one contiguous run.
#include <array>
#include <cmath>

#include "cplx.cuh"
#include "rf_internal.h"

namespace rf {

namespace {

template <typename V, int R, int SIGN>
__global__ void __launch_bounds__(256) k_stockham(const V* __restrict__ in, V* __restrict__ out,
                                                  int64_t n, int64_t Ns, const V* __restrict__ tw,
                                                  int64_t tw_stride) {
  const int64_t nb = n / R;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  const int64_t row = (int64_t)blockIdx.y * n;
  in += row;
  out += row;
  const int64_t k = j & (Ns - 1);
  V a[R];
#pragma unroll
  for (int t = 0; t < R; ++t) a[t] = in[j + t * nb];
  if (Ns > 1) {
    // w^(t k) = exp(sign 2 pi i t k / (Ns R)) = table[t k (n / (Ns R))] (conjugated for sign +1)
    const int64_t step = (n / (Ns * R)) * tw_stride;
#pragma unroll
    for (int t = 1; t < R; ++t) a[t] = tw_apply<SIGN>(a[t], tw[(int64_t)t * k * step]);
  }
  dft<R, SIGN>(a);
  const int64_t base = (j - k) * R + k;
#pragma unroll
  for (int t = 0; t < R; ++t) out[base + t * Ns] = a[t];
}

// First pass of a transform whose input is the one-sided product X[k] F[k] for k <= n/2 and
// zero above (the matched-filter integrand of Eq. 2): the product is formed on load.
template <typename V, int R, int SIGN>
__global__ void __launch_bounds__(256) k_stockham_first_mul(const V* __restrict__ X, const V* __restrict__ F,
                                                            int64_t fstride, V* __restrict__ out, int64_t n) {
  const int64_t nb = n / R;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  F += (int64_t)blockIdx.y * fstride;
  out += (int64_t)blockIdx.y * n;
  const int64_t half = n / 2;
  V a[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int64_t k = j + t * nb;
    a[t] = k <= half ? cmul(X[k], F[k]) : cmake<V>(0, 0);
  }
  dft<R, SIGN>(a);
#pragma unroll
  for (int t = 0; t < R; ++t) out[j * R + t] = a[t];
}

template <typename V, int R>
void launch_pass(const V* in, V* out, int64_t n, int64_t Ns, int batch, int sign, const V* tw,
                 int64_t tw_stride, cudaStream_t s) {
  const int64_t nb = n / R;
  dim3 block(256);
  dim3 grid((unsigned)((nb + 255) / 256), (unsigned)batch);
  if (sign < 0)
    k_stockham<V, R, -1><<<grid, block, 0, s>>>(in, out, n, Ns, tw, tw_stride);
  else
    k_stockham<V, R, +1><<<grid, block, 0, s>>>(in, out, n, Ns, tw, tw_stride);
  RF_LAUNCHED();
}

template <typename V>
void fft_c2c(const V* in, V* out, V* tmp, int64_t n, int batch, int sign, const V* tw,
             int64_t table_n, cudaStream_t s, const V* mulF = nullptr, int64_t fstride = 0) {
  RF_REQUIRE(n >= 2 && (n & (n - 1)) == 0, "fft: n=%lld is not a power of two", (long long)n);
  RF_REQUIRE(table_n % n == 0, "fft: twiddle table too small");
  RF_REQUIRE(batch >= 1 && batch <= 65535, "fft: batch %d out of range", batch);
  RF_REQUIRE(in != out && in != tmp && out != tmp, "fft: buffers must be distinct");
  int bits = 0;
  while ((int64_t(1) << bits) < n) ++bits;
  // pass radices in a fixed array (no host allocation per call): n < 2^40 needs at most 10
  std::array<int, 10> radix{};
  int P = 0;
  RF_REQUIRE(bits < 40, "fft: n=%lld is too large", (long long)n);
  while (bits >= 4) {
    radix[P++] = 16;
    bits -= 4;
  }
  if (bits) radix[P++] = 1 << bits;
  const int64_t tw_stride = table_n / n;
  const V* src = in;
  int64_t Ns = 1;
  for (int p = 0; p < P; ++p) {
    V* dst = ((P - 1 - p) % 2 == 0) ? out : tmp;
    if (p == 0 && mulF) {
      RF_REQUIRE(radix[0] == 16 && sign > 0, "fft: the product pass needs n >= 16 and an inverse transform");
      dim3 grid((unsigned)((n / 16 + 255) / 256), (unsigned)batch);
      k_stockham_first_mul<V, 16, +1><<<grid, 256, 0, s>>>(in, mulF, fstride, dst, n);
      RF_LAUNCHED();
      Ns *= radix[p];
      src = dst;
      continue;
    }
    switch (radix[p]) {
      case 16: launch_pass<V, 16>(src, dst, n, Ns, batch, sign, tw, tw_stride, s); break;
      case 8: launch_pass<V, 8>(src, dst, n, Ns, batch, sign, tw, tw_stride, s); break;
      case 4: launch_pass<V, 4>(src, dst, n, Ns, batch, sign, tw, tw_stride, s); break;
      default: launch_pass<V, 2>(src, dst, n, Ns, batch, sign, tw, tw_stride, s); break;
    }
    Ns *= radix[p];
    src = dst;
  }
}

template <typename T, typename V>
__global__ void k_real_to_complex(const T* __restrict__ x, V* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = cmake<V>(x[i], (T)0);
}

}  // namespace

void fft_c2c_f64(const double2* in, double2* out, double2* tmp, int64_t n, int batch, int sign,
                 const double2* tw, int64_t table_n, cudaStream_t s) {
  fft_c2c<double2>(in, out, tmp, n, batch, sign, tw, table_n, s);
}

void fft_c2c_f32(const float2* in, float2* out, float2* tmp, int64_t n, int batch, int sign,
                 const float2* tw, int64_t table_n, cudaStream_t s) {
  fft_c2c<float2>(in, out, tmp, n, batch, sign, tw, table_n, s);
}

void ifft_product_f64(const double2* X, const double2* F, int64_t fstride, double2* out, double2* tmp, int64_t n,
                      int batch, const double2* tw, int64_t table_n, cudaStream_t s) {
  fft_c2c<double2>(X, out, tmp, n, batch, +1, tw, table_n, s, F, fstride);
}

void ifft_product_f32(const float2* X, const float2* F, int64_t fstride, float2* out, float2* tmp, int64_t n,
                      int batch, const float2* tw, int64_t table_n, cudaStream_t s) {
  fft_c2c<float2>(X, out, tmp, n, batch, +1, tw, table_n, s, F, fstride);
}

void real_to_complex_f64(const double* x, double2* out, int64_t n, cudaStream_t s) {
  k_real_to_complex<double, double2><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, out, n);
  RF_LAUNCHED();
}

void real_to_complex_f32(const float* x, float2* out, int64_t n, cudaStream_t s) {
  k_real_to_complex<float, float2><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, out, n);
  RF_LAUNCHED();
}

std::vector<double2> host_twiddles(int64_t n) {
  // exp(-2 pi i m / n) for m < n.  Angles are reduced to the first octant, where
  // cos and sin are evaluated directly; the other octants follow by exact symmetry.
  std::vector<double2> w((size_t)n);
  const double two_pi = 6.283185307179586476925286766559;
  for (int64_t m = 0; m < n; ++m) {
    // angle = 2 pi m / n = (pi/4) (octant + frac)
    const int64_t e = m * 8;  // in units of 2 pi / (8 n) ... position in eighths of a turn
    const int64_t oct = e / n;
    const int64_t rem = e - oct * n;  // angle within the octant = (pi/4) rem / n
    double c, s;
    auto cs = [&](int64_t r, double& cc, double& ss) {
      const double a = two_pi * (double)r / (8.0 * (double)n);
      cc = std::cos(a);
      ss = std::sin(a);
    };
    switch (oct) {
      case 0: cs(rem, c, s); break;
      case 1: { double cc, ss; cs(n - rem, cc, ss); c = ss; s = cc; } break;
      case 2: { double cc, ss; cs(rem, cc, ss); c = -ss; s = cc; } break;
      case 3: { double cc, ss; cs(n - rem, cc, ss); c = -cc; s = ss; } break;
      case 4: { double cc, ss; cs(rem, cc, ss); c = -cc; s = -ss; } break;
      case 5: { double cc, ss; cs(n - rem, cc, ss); c = -ss; s = -cc; } break;
      case 6: { double cc, ss; cs(rem, cc, ss); c = ss; s = -cc; } break;
      default: { double cc, ss; cs(n - rem, cc, ss); c = cc; s = -ss; } break;
    }
    // (c, s) = (cos, sin)(2 pi m / n); the table holds exp(-i angle)
    w[(size_t)m] = make_double2(c, -s);
  }
  return w;
}

}  // namespace rf
