// Reference matched filter (Sec. II.A, Eqs. 2-4 and 6) and template spectra.
#include <cmath>

#include "cplx.cuh"
#include "rf_internal.h"
#include "tf2.cuh"

namespace rf {

Tf2 make_tf2(const rf_template& t, int pn_order) {
  // Non-spinning TaylorF2 coefficients (Buonanno, Iyer, Ochsner, Pan & Sathyaprakash 2009),
  // truncated at v^pn_order.
  const double msun_s = 4.925491025543576e-6;
  const double pi = kPi;
  const double gamma_e = 0.57721566490153286061;
  Tf2 p{};
  const double mt = t.m1 + t.m2;
  p.M = mt * msun_s;
  p.eta = t.m1 * t.m2 / (mt * mt);
  p.tc = t.tc;
  p.phic = t.phic;
  p.pref = 3.0 / (128.0 * p.eta);
  const double e = p.eta;
  for (double& a : p.a) a = 0.0;
  p.a[0] = 1.0;
  if (pn_order >= 2) p.a[2] = 3715.0 / 756.0 + 55.0 / 9.0 * e;
  if (pn_order >= 3) p.a[3] = -16.0 * pi;
  if (pn_order >= 4) p.a[4] = 15293365.0 / 508032.0 + 27145.0 / 504.0 * e + 3085.0 / 72.0 * e * e;
  if (pn_order >= 5) {
    const double a5 = pi * (38645.0 / 756.0 - 65.0 / 9.0 * e);
    p.a[5] = a5;
    p.a5log = 3.0 * a5;
  }
  if (pn_order >= 6) {
    p.a[6] = 11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * pi * pi - 6848.0 / 21.0 * gamma_e +
             (-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * pi * pi) * e + 76055.0 / 1728.0 * e * e -
             127825.0 / 1296.0 * e * e * e;
    p.a6log = -6848.0 / 21.0;
  }
  if (pn_order >= 7) p.a[7] = pi * (77096675.0 / 254016.0 + 378515.0 / 1512.0 * e - 74045.0 / 756.0 * e * e);
  return p;
}

namespace {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 512;

// Partial sums of 4 df B(f_k)^2 inv_psd[k] over the band, one partial per block.
__global__ void __launch_bounds__(kRedThreads) k_sigma2_partial(const double* __restrict__ ip, int64_t nbins,
                                                                double df, double f_low, double f_high,
                                                                double* __restrict__ part) {
  double acc = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nbins;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double f = (double)k * df;
    if (f >= f_low && f <= f_high && k > 0) acc += exp(-7.0 / 3.0 * log(f)) * ip[k];
  }
  __shared__ double sh[kRedThreads];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = 4.0 * df * sh[0];
}

__global__ void k_sum_partials(const double* __restrict__ part, int count, double* __restrict__ out) {
  __shared__ double sh[kRedThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += part[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

// Z~[k] = (4 / (n N)) X[k] conj(h~_k) inv_psd[k] on the band, 0 elsewhere and for k > n/2.
// X is the unnormalised DFT of the data (x~ = dt X), so 4 df dt = 4 / n.
template <typename V>
__global__ void __launch_bounds__(256) k_mf_pointwise(const V* __restrict__ X, const double* __restrict__ ip,
                                                      const double* __restrict__ sigma2, Tf2 p, int64_t n,
                                                      double df, double f_low, double f_high, V* __restrict__ Z,
                                                      double* __restrict__ sigma_out) {
  using R = typename real_of<V>::type;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0 && sigma_out) sigma_out[0] = sqrt(sigma2[0]);
  if (k >= n) return;
  const double f = (double)k * df;
  V out = cmake<V>((R)0, (R)0);
  if (k <= n / 2 && k > 0 && f >= f_low && f <= f_high) {
    const double psi = tf2_phase(p, f);
    const double scale = 4.0 / ((double)n * sqrt(sigma2[0]));
    if constexpr (sizeof(R) == 8) {
      double s, c;
      sincos(psi, &s, &c);
      const double a = scale * tf2_amp(f) * ip[k];
      // conj(h~) = B exp(+i Psi)
      out = cmul(X[k], cmake<V>(a * c, a * s));
    } else {
      // reduce the FP64 phase to (-pi, pi] before the FP32 sine/cosine
      const double red = psi - kTwoPi * rint(psi * (1.0 / kTwoPi));
      float s, c;
      sincosf((float)red, &s, &c);
      const float a = (float)(scale * ip[k]) * powf((float)f, -7.0f / 6.0f);
      out = cmul(X[k], cmake<V>(a * c, a * s));
    }
  }
  Z[k] = out;
}

template <typename V>
__global__ void __launch_bounds__(256) k_template_fd(Tf2 p, int64_t nbins, double df, V* __restrict__ h) {
  using R = typename real_of<V>::type;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nbins) return;
  V out = cmake<V>((R)0, (R)0);
  if (k > 0) {
    const double f = (double)k * df;
    const double psi = tf2_phase(p, f);
    double s, c;
    sincos(psi, &s, &c);
    const double a = tf2_amp(f);
    out = cmake<V>((R)(a * c), (R)(-a * s));
  }
  h[k] = out;
}

}  // namespace

void sigma2_impl(rf_ctx* c, const double* inv_psd, int count, double* out, cudaStream_t s) {
  const int64_t nbins = c->n / 2 + 1;
  c->red.ensure(sizeof(double) * kRedBlocks);
  double* part = c->red.as<double>();
  const double df = c->g.fs / (double)c->n;
  k_sigma2_partial<<<kRedBlocks, kRedThreads, 0, s>>>(inv_psd, nbins, df, c->g.f_low, c->g.f_high, part);
  RF_LAUNCHED();
  for (int i = 0; i < count; ++i) {
    k_sum_partials<<<1, kRedThreads, 0, s>>>(part, kRedBlocks, out + i);
    RF_LAUNCHED();
  }
}

void mf_reference_impl(rf_ctx* c, const void* x, const double* inv_psd, int32_t nref, const rf_template* refs,
                       void* z_out, double* sigma_out, cudaStream_t s) {
  const int64_t n = c->n;
  const double df = c->g.fs / (double)n;
  // sigma^2 is the same for every template of the unit-amplitude family (B = f^-7/6);
  // it is computed once per call in FP64 (Eq. 3) and kept after the partials.
  c->red.ensure(sizeof(double) * (kRedBlocks + 8));
  double* sig2 = c->red.as<double>() + kRedBlocks;
  {
    const int64_t nbins = n / 2 + 1;
    k_sigma2_partial<<<kRedBlocks, kRedThreads, 0, s>>>(inv_psd, nbins, df, c->g.f_low, c->g.f_high,
                                                       c->red.as<double>());
    RF_LAUNCHED();
    k_sum_partials<<<1, kRedThreads, 0, s>>>(c->red.as<double>(), kRedBlocks, sig2);
    RF_LAUNCHED();
  }
  const unsigned grid = (unsigned)((n + 255) / 256);
  if (c->g.dtype == RF_F64) {
    real_to_complex_f64(static_cast<const double*>(x), c->fa.as<double2>(), n, s);
    fft_c2c_f64(c->fa.as<double2>(), c->xf.as<double2>(), c->fb.as<double2>(), n, 1, -1, c->tw64.as<double2>(), n,
                s);
    for (int r = 0; r < nref; ++r) {
      const Tf2 p = make_tf2(refs[r], c->g.pn_order);
      k_mf_pointwise<double2><<<grid, 256, 0, s>>>(c->xf.as<double2>(), inv_psd, sig2, p, n, df, c->g.f_low,
                                                   c->g.f_high, c->fa.as<double2>(), sigma_out ? sigma_out + r : nullptr);
      RF_LAUNCHED();
      fft_c2c_f64(c->fa.as<double2>(), static_cast<double2*>(z_out) + (int64_t)r * n, c->fb.as<double2>(), n, 1,
                  +1, c->tw64.as<double2>(), n, s);
    }
  } else {
    real_to_complex_f32(static_cast<const float*>(x), c->fa.as<float2>(), n, s);
    fft_c2c_f32(c->fa.as<float2>(), c->xf.as<float2>(), c->fb.as<float2>(), n, 1, -1, c->tw32.as<float2>(), n, s);
    for (int r = 0; r < nref; ++r) {
      const Tf2 p = make_tf2(refs[r], c->g.pn_order);
      k_mf_pointwise<float2><<<grid, 256, 0, s>>>(c->xf.as<float2>(), inv_psd, sig2, p, n, df, c->g.f_low,
                                                  c->g.f_high, c->fa.as<float2>(), sigma_out ? sigma_out + r : nullptr);
      RF_LAUNCHED();
      fft_c2c_f32(c->fa.as<float2>(), static_cast<float2*>(z_out) + (int64_t)r * n, c->fb.as<float2>(), n, 1, +1,
                  c->tw32.as<float2>(), n, s);
    }
  }
}

void template_fd_impl(rf_ctx* c, const rf_template& t, void* h_out, cudaStream_t s) {
  const int64_t nbins = c->n / 2 + 1;
  const double df = c->g.fs / (double)c->n;
  const Tf2 p = make_tf2(t, c->g.pn_order);
  const unsigned grid = (unsigned)((nbins + 255) / 256);
  if (c->g.dtype == RF_F64)
    k_template_fd<double2><<<grid, 256, 0, s>>>(p, nbins, df, static_cast<double2*>(h_out));
  else
    k_template_fd<float2><<<grid, 256, 0, s>>>(p, nbins, df, static_cast<float2*>(h_out));
  RF_LAUNCHED();
}

}  // namespace rf
