// Reference matched filter (Sec. II.A, Eqs. 2-4 and 6) and template spectra.
#include <algorithm>
#include <cmath>
#include <mutex>

#include <cuda.h>

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
// complex values of the four-step inverse transforms launched together (their intermediate)
constexpr int64_t kF4Chunk = int64_t(1) << 23;

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

// Stored reference filter: F[k] = (4 / (n N)) conj(h~_k) inv_psd[k] on the band, 0 elsewhere,
// k = 0..n/2, phase and scale in FP64 and rounded once.  With X the unnormalised DFT of the
// data, X[k] F[k] is the integrand of Eq. 2 (4 df dt = 4 / n).
template <typename V>
__global__ void __launch_bounds__(256) k_ref_filter(const double* __restrict__ ip, const double* __restrict__ sigma2,
                                                    Tf2 p, int64_t n, double df, double f_low, double f_high,
                                                    V* __restrict__ F, double* __restrict__ sigma_out) {
  using R = typename real_of<V>::type;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0 && sigma_out) sigma_out[0] = sqrt(sigma2[0]);
  if (k > n / 2) return;
  const double f = (double)k * df;
  V out = cmake<V>((R)0, (R)0);
  if (k > 0 && f >= f_low && f <= f_high) {
    double sn, cs;
    sincos(tf2_phase(p, f), &sn, &cs);
    const double a = 4.0 / ((double)n * sqrt(sigma2[0])) * tf2_amp(f) * ip[k];
    out = cmake<V>((R)(a * cs), (R)(a * sn));  // conj(h~) = B exp(+i Psi)
  }
  F[k] = out;
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
    const bool four = fft4_supported(n);  // two-pass four-step transforms, else radix passes
    if (four) {
      fft4_forward_real(c, static_cast<const float*>(x), c->xf.as<float2>(), c->fb.as<float2>(), s);
    } else {
      real_to_complex_f32(static_cast<const float*>(x), c->fa.as<float2>(), n, s);
      fft_c2c_f32(c->fa.as<float2>(), c->xf.as<float2>(), c->fb.as<float2>(), n, 1, -1, c->tw32.as<float2>(), n,
                  s);
    }
    for (int r = 0; r < nref; ++r) {
      const Tf2 p = make_tf2(refs[r], c->g.pn_order);
      k_mf_pointwise<float2><<<grid, 256, 0, s>>>(c->xf.as<float2>(), inv_psd, sig2, p, n, df, c->g.f_low,
                                                  c->g.f_high, c->fa.as<float2>(), sigma_out ? sigma_out + r : nullptr);
      RF_LAUNCHED();
      float2* zr = static_cast<float2*>(z_out) + (int64_t)r * n;
      if (four)
        fft4_inverse(c, c->fa.as<float2>(), zr, c->fb.as<float2>(), 1, s);
      else
        fft_c2c_f32(c->fa.as<float2>(), zr, c->fb.as<float2>(), n, 1, +1, c->tw32.as<float2>(), n, s);
    }
  }
}

void reference_filters_impl(rf_ctx* c, const double* inv_psd, int32_t nref, const rf_template* refs, void* filt,
                            double* sigma_out, cudaStream_t s) {
  const int64_t n = c->n;
  const int64_t nb = n / 2 + 1;
  const double df = c->g.fs / (double)n;
  c->red.ensure(sizeof(double) * (kRedBlocks + 8));
  double* sig2 = c->red.as<double>() + kRedBlocks;
  k_sigma2_partial<<<kRedBlocks, kRedThreads, 0, s>>>(inv_psd, nb, df, c->g.f_low, c->g.f_high, c->red.as<double>());
  RF_LAUNCHED();
  k_sum_partials<<<1, kRedThreads, 0, s>>>(c->red.as<double>(), kRedBlocks, sig2);
  RF_LAUNCHED();
  const unsigned grid = (unsigned)((nb + 255) / 256);
  for (int r = 0; r < nref; ++r) {
    const Tf2 p = make_tf2(refs[r], c->g.pn_order);
    double* so = sigma_out ? sigma_out + r : nullptr;
    if (c->g.dtype == RF_F64)
      k_ref_filter<double2><<<grid, 256, 0, s>>>(inv_psd, sig2, p, n, df, c->g.f_low, c->g.f_high,
                                                 static_cast<double2*>(filt) + (int64_t)r * nb, so);
    else
      k_ref_filter<float2><<<grid, 256, 0, s>>>(inv_psd, sig2, p, n, df, c->g.f_low, c->g.f_high,
                                                static_cast<float2*>(filt) + (int64_t)r * nb, so);
    RF_LAUNCHED();
  }
}

void mf_filtered_impl(rf_ctx* c, const void* x, int32_t nref, const void* filt, void* z_out, cudaStream_t s) {
  const int64_t n = c->n;
  const int64_t nb = n / 2 + 1;
  // references per batched inverse transform, bounded by the temporary buffer
  const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(nref, std::min<int64_t>(65535, (int64_t)(1 << 27) / n)));
  if (c->g.dtype == RF_F64) {
    c->mf_tmp.ensure(sizeof(double2) * (size_t)chunk * n);
    real_to_complex_f64(static_cast<const double*>(x), c->fa.as<double2>(), n, s);
    fft_c2c_f64(c->fa.as<double2>(), c->xf.as<double2>(), c->fb.as<double2>(), n, 1, -1, c->tw64.as<double2>(), n,
                s);
    for (int r0 = 0; r0 < nref; r0 += chunk) {
      const int cnt = std::min(chunk, nref - r0);
      ifft_product_f64(c->xf.as<double2>(), static_cast<const double2*>(filt) + (int64_t)r0 * nb, nb,
                       static_cast<double2*>(z_out) + (int64_t)r0 * n, c->mf_tmp.as<double2>(), n, cnt,
                       c->tw64.as<double2>(), n, s);
    }
  } else if (fft4_supported(n)) {
    // two-pass four-step transforms; the inverses of kF4Chunk references share one launch pair,
    // whose intermediate (kF4Chunk n complex values) is meant to stay in L2
    const int c4 = (int)std::min<int64_t>(nref, std::max<int64_t>(1, kF4Chunk / n));
    c->mf_tmp.ensure(sizeof(float2) * (size_t)c4 * n);
    fft4_forward_real(c, static_cast<const float*>(x), c->xf.as<float2>(), c->mf_tmp.as<float2>(), s);
    for (int r0 = 0; r0 < nref; r0 += c4) {
      const int cnt = std::min(c4, nref - r0);
      fft4_inverse_product(c, c->xf.as<float2>(), static_cast<const float2*>(filt) + (int64_t)r0 * nb, nb,
                           static_cast<float2*>(z_out) + (int64_t)r0 * n, c->mf_tmp.as<float2>(), cnt, s);
    }
  } else {
    c->mf_tmp.ensure(sizeof(float2) * (size_t)chunk * n);
    real_to_complex_f32(static_cast<const float*>(x), c->fa.as<float2>(), n, s);
    fft_c2c_f32(c->fa.as<float2>(), c->xf.as<float2>(), c->fb.as<float2>(), n, 1, -1, c->tw32.as<float2>(), n, s);
    for (int r0 = 0; r0 < nref; r0 += chunk) {
      const int cnt = std::min(chunk, nref - r0);
      ifft_product_f32(c->xf.as<float2>(), static_cast<const float2*>(filt) + (int64_t)r0 * nb, nb,
                       static_cast<float2*>(z_out) + (int64_t)r0 * n, c->mf_tmp.as<float2>(), n, cnt,
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

// ---------------------------------------------------------------- allocation-free variant
// rf_mf_reference_noalloc: the reference matched filter for callers that may not
// allocate device memory.  Its workspace is the file-scope array below (about
// 4 MiB, reserved in every GPU that loads the library, until the process exits).

namespace {

constexpr int64_t kNoAllocMaxN = int64_t(1) << 16;
constexpr size_t kNoAllocSlot = (size_t)kNoAllocMaxN * sizeof(double2);  // one complex128 row of kNoAllocMaxN
constexpr size_t kNoAllocRed = 8192;                                      // FP64 partial sums + sigma^2
constexpr size_t kNoAllocBytes = 4 * kNoAllocSlot + kNoAllocRed;
// The array has its own device address in every CUDA context that loads the module (the
// runtime's primary context of each device, or a context a host application created with
// the driver API), so the addresses are remembered per context, keyed by the context's
// process-unique ID (a handle value can be reused by a later context; the ID is not).
constexpr int kNoAllocCacheSlots = 64;
struct NoAllocSlot {
  unsigned long long ctx_id;
  void* addr;
};
std::mutex g_noalloc_mu;
NoAllocSlot g_noalloc_cache[kNoAllocCacheSlots] = {};
int g_noalloc_used = 0;
int g_noalloc_next = 0;

// exp(-2 pi i m / n), m < n, into the workspace (rebuilt on every call).
template <typename V>
__global__ void __launch_bounds__(256) k_noalloc_twiddles(V* __restrict__ tw, int64_t n) {
  using R = typename real_of<V>::type;
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  double s, c;
  sincospi(2.0 * (double)m / (double)n, &s, &c);
  tw[m] = cmake<V>((R)c, (R)(-s));
}

}  // namespace

}  // namespace rf

// The workspace.  Host code must not use this name as an address: it is a host-side
// stand-in.  The device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char rf_noalloc_scratch[rf::kNoAllocBytes];

namespace rf {
namespace {

// Driver entry points for the current context and its ID, looked up once through the
// runtime (no link against the driver library).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

struct CtxFns {
  CtxGetCurrentFn get_current;
  CtxGetIdFn get_id;
};

const CtxFns& ctx_fns() {
  static const CtxFns fns = [] {
    CtxFns f{nullptr, nullptr};
    void* a = nullptr;
    void* b = nullptr;
    cudaDriverEntryPointQueryResult qa{}, qb{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 4000, cudaEnableDefault, &qa) == cudaSuccess &&
        qa == cudaDriverEntryPointSuccess)
      f.get_current = reinterpret_cast<CtxGetCurrentFn>(a);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
        qb == cudaDriverEntryPointSuccess)
      f.get_id = reinterpret_cast<CtxGetIdFn>(b);
    (void)cudaGetLastError();
    return f;
  }();
  return fns;
}

// Process-unique ID of the calling thread's current context, or 0 when none is current.
unsigned long long current_context_id() {
  const CtxFns& f = ctx_fns();
  RF_REQUIRE(f.get_current != nullptr && f.get_id != nullptr,
             "the driver does not provide cuCtxGetCurrent / cuCtxGetId");
  CUcontext ctx = nullptr;
  if (f.get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return 0;
  unsigned long long id = 0;
  RF_REQUIRE(f.get_id(ctx, &id) == CUDA_SUCCESS, "cuCtxGetId failed on the current context");
  return id;
}

void* lookup_scratch_symbol() {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, rf_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr) {
    (void)cudaGetLastError();
    set_error("cudaGetSymbolAddress of the static workspace failed: %s", cudaGetErrorString(e));
    throw Fail{RF_ECUDA};
  }
  return p;
}

// Device address of rf_noalloc_scratch in the calling thread's current context.  The
// set-up (cudaGetSymbolAddress) runs on the first call made in a context and its result is
// remembered for that context; a thread with no current context gets the runtime's
// primary context of its current device, which that first runtime call binds.
unsigned char* noalloc_scratch_address() {
  unsigned long long id = current_context_id();
  void* fresh = nullptr;
  if (id == 0) {
    fresh = lookup_scratch_symbol();  // binds the primary context
    id = current_context_id();
    RF_REQUIRE(id != 0, "no CUDA context is current after the workspace lookup");
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  for (int i = 0; i < g_noalloc_used; ++i)
    if (g_noalloc_cache[i].ctx_id == id) return static_cast<unsigned char*>(g_noalloc_cache[i].addr);
  if (!fresh) fresh = lookup_scratch_symbol();
  // remember it; with every slot taken, the oldest entry makes room
  int slot;
  if (g_noalloc_used < kNoAllocCacheSlots) {
    slot = g_noalloc_used++;
  } else {
    slot = g_noalloc_next;
    g_noalloc_next = (g_noalloc_next + 1) % kNoAllocCacheSlots;
  }
  g_noalloc_cache[slot] = NoAllocSlot{id, fresh};
  return static_cast<unsigned char*>(fresh);
}

void noalloc_check_dev(const void* p, const char* name, bool allow_null) {
  if (!p) {
    RF_REQUIRE(allow_null, "%s is NULL", name);
    return;
  }
  RF_REQUIRE(((uintptr_t)p & 15u) == 0, "%s is not 16-byte aligned", name);
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    RF_REQUIRE(false, "%s is not a CUDA device pointer", name);
  }
  RF_REQUIRE(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged, "%s is not device memory", name);
}

void mf_reference_noalloc_impl(const rf_grid& g, const void* x, const double* inv_psd, const rf_template& ref,
                               void* z_out, double* sigma_out, cudaStream_t s) {
  RF_REQUIRE(g.n >= 256 && (g.n & (g.n - 1)) == 0, "n=%lld must be a power of two >= 256", (long long)g.n);
  RF_REQUIRE(g.n <= kNoAllocMaxN, "n=%lld exceeds the static workspace limit n <= %lld of rf_mf_reference_noalloc",
             (long long)g.n, (long long)kNoAllocMaxN);
  RF_REQUIRE(std::isfinite(g.fs) && g.fs > 0, "fs must be positive");
  RF_REQUIRE(std::isfinite(g.f_low) && std::isfinite(g.f_high) && g.f_low > 0 && g.f_low < g.f_high,
             "need 0 < f_low < f_high");
  RF_REQUIRE(g.f_high + g.df_high <= 0.5 * g.fs * (1 + 1e-12) && g.df_high >= 0,
             "f_high + df_high must not exceed fs/2");
  RF_REQUIRE(g.pn_order >= 0 && g.pn_order <= 7, "pn_order must be 0..7");
  RF_REQUIRE(g.dtype == RF_F64 || g.dtype == RF_F32, "dtype must be RF_F64 or RF_F32");
  RF_REQUIRE(std::isfinite(ref.m1) && std::isfinite(ref.m2) && ref.m1 > 0 && ref.m2 > 0 && std::isfinite(ref.tc) &&
                 std::isfinite(ref.phic),
             "ref: masses must be positive and all fields finite");
  noalloc_check_dev(x, "x", false);
  noalloc_check_dev(inv_psd, "inv_psd", false);
  noalloc_check_dev(z_out, "z_out", false);
  noalloc_check_dev(sigma_out, "sigma_out", true);

  unsigned char* ws = noalloc_scratch_address();
  const int64_t n = g.n;
  const double df = g.fs / (double)n;
  void* tw = ws;
  void* xf = ws + kNoAllocSlot;
  void* fa = ws + 2 * kNoAllocSlot;
  void* fb = ws + 3 * kNoAllocSlot;
  double* part = reinterpret_cast<double*>(ws + 4 * kNoAllocSlot);
  double* sig2 = part + kRedBlocks;
  static_assert((kRedBlocks + 1) * sizeof(double) <= kNoAllocRed, "reduction slots");
  // Every region is fully rewritten below before it is read (twiddles, spectra, partial
  // sums), so nothing left by an earlier call leaks into this one.
  const unsigned grid = (unsigned)((n + 255) / 256);
  k_sigma2_partial<<<kRedBlocks, kRedThreads, 0, s>>>(inv_psd, n / 2 + 1, df, g.f_low, g.f_high, part);
  RF_LAUNCHED();
  k_sum_partials<<<1, kRedThreads, 0, s>>>(part, kRedBlocks, sig2);
  RF_LAUNCHED();
  const Tf2 p = make_tf2(ref, g.pn_order);
  if (g.dtype == RF_F64) {
    k_noalloc_twiddles<double2><<<grid, 256, 0, s>>>(static_cast<double2*>(tw), n);
    RF_LAUNCHED();
    real_to_complex_f64(static_cast<const double*>(x), static_cast<double2*>(fa), n, s);
    fft_c2c_f64(static_cast<double2*>(fa), static_cast<double2*>(xf), static_cast<double2*>(fb), n, 1, -1,
                static_cast<double2*>(tw), n, s);
    k_mf_pointwise<double2><<<grid, 256, 0, s>>>(static_cast<double2*>(xf), inv_psd, sig2, p, n, df, g.f_low,
                                                 g.f_high, static_cast<double2*>(fa), sigma_out);
    RF_LAUNCHED();
    fft_c2c_f64(static_cast<double2*>(fa), static_cast<double2*>(z_out), static_cast<double2*>(fb), n, 1, +1,
                static_cast<double2*>(tw), n, s);
  } else {
    k_noalloc_twiddles<float2><<<grid, 256, 0, s>>>(static_cast<float2*>(tw), n);
    RF_LAUNCHED();
    real_to_complex_f32(static_cast<const float*>(x), static_cast<float2*>(fa), n, s);
    fft_c2c_f32(static_cast<float2*>(fa), static_cast<float2*>(xf), static_cast<float2*>(fb), n, 1, -1,
                static_cast<float2*>(tw), n, s);
    k_mf_pointwise<float2><<<grid, 256, 0, s>>>(static_cast<float2*>(xf), inv_psd, sig2, p, n, df, g.f_low,
                                                g.f_high, static_cast<float2*>(fa), sigma_out);
    RF_LAUNCHED();
    fft_c2c_f32(static_cast<float2*>(fa), static_cast<float2*>(z_out), static_cast<float2*>(fb), n, 1, +1,
                static_cast<float2*>(tw), n, s);
  }
}

}  // namespace
}  // namespace rf

extern "C" rf_status rf_mf_reference_noalloc(const rf_grid* grid, const void* x, const double* inv_psd,
                                             const rf_template* ref, void* z_out, double* sigma_out,
                                             rf_stream stream) {
  rf::clear_error();
  try {
    RF_REQUIRE(grid != nullptr && ref != nullptr, "grid and ref must be non-NULL");
    rf::mf_reference_noalloc_impl(*grid, x, inv_psd, *ref, z_out, sigma_out, (cudaStream_t)stream);
    return RF_OK;
  } catch (const rf::Fail& e) {
    return e.st;
  } catch (...) {
    rf::set_error("unexpected internal error");
    return RF_EINVAL;
  }
}
