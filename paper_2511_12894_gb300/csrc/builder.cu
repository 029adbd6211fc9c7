// Ratio-kernel builder (Sec. II.B-II.D; Eqs. 5, 7, 9, 10), FP64 throughout.
//
// Per neighbour j of the reference, on its build grid of n_b bins (f_k = k fs / n_b; n_b = n
// unless a coarser grid is asked for, Sec. II.D):
//   df_low_j = min(df_low_max, f_low / 2, 1 / sqrt(|dPsi''(f_low)| / (2 pi)))          (Eq. 10)
//   K~_j[k]  = (N_ref / N_j) R(f_k) W_j(f_k) exp(+i (Psi_j(f_k) - Psi_ref(f_k))) / n_b   (Eqs. 5, 7, 9)
//   rho_j    = unnormalised n_b-point inverse DFT of K~_j (zero for k > n_b/2)
//   kept     = { m : |rho_j[m]|^2 >= thr^2 a_j },  a_j = max |rho_j|^2 (relative) or 1
//   [m0, m0 + L) = shortest circular arc covering `kept`, ties to the smallest signed m0
//   taps c_j[l] = rho_j[(m0 + l) mod n_b]
// The automatic grid is the smallest power of two of at least four times the lag extent
// between the time offsets dt(f) = (Psi_j' - Psi_ref')(f) / (2 pi) (Eq. A2) at the window
// edges f_low - df_low_j and f_high + df_high, plus the taper spread 4 fs / df_low_j
// (capped at n); neighbours are processed grouped by grid.
// The templates share the amplitude law B = f^-7/6, so R = 1 and N_ref / N_j = 1;
// both factors are still formed from their definitions.
#include <algorithm>
#include <climits>
#include <cmath>
#include <memory>

#include "cplx.cuh"
#include "rf_internal.h"
#include "tf2.cuh"

namespace rf {

namespace {

__global__ void k_df_low(Tf2 ref, const Tf2* __restrict__ tg, int count, double f_low, double df_low_max,
                         double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= count) return;
  const double d2 = tf2_d2phase(tg[j], f_low) - tf2_d2phase(ref, f_low);
  const double dtp = fabs(d2) / kTwoPi;  // |d t'(f_low)| = |d tau'(f_low)| for a common t_c
  double v = fmin(df_low_max, 0.5 * f_low);
  if (dtp > 0.0) v = fmin(v, 1.0 / sqrt(dtp));
  out[j] = v;
}

// Lag extent of each kernel for the automatic build grid (samples).
__global__ void k_grid_extent(Tf2 ref, const Tf2* __restrict__ tg, const double* __restrict__ dfl, int count,
                              double fs, double f_low, double f_high, double df_high, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= count) return;
  const double fa = f_low - dfl[j], fb = f_high + df_high;
  const double ta = (tf2_dphase(tg[j], fa) - tf2_dphase(ref, fa)) / kTwoPi;
  const double tb = (tf2_dphase(tg[j], fb) - tf2_dphase(ref, fb)) / kTwoPi;
  out[j] = fmax(fabs(ta), fabs(tb)) * fs + 4.0 * fs / dfl[j];
}

// Analytic truncation (Sec. II.D with the App. A expressions), one thread per template: the
// threshold amplitude A on |r| = 2 fs |rho| (N_ref / N_j = 1: one amplitude law) is thr times
// the kernel's peak (relative) or thr; each taper end f_e reaches d_e = (R / (4 pi df_e^2 A))^(1/3)
// on both sides of its lag time c_e = -dt(f_e); the kept lags run from floor(min(c_e - d_e) fs)
// to ceil(max(c_e + d_e) fs), at most the grid.
// (rfac: |r| = rfac fs |rho|, 2 for the complex kernel, 1 for the real form's taps 2 Re rho.)
__global__ void k_analytic_span(Tf2 ref, const Tf2* __restrict__ tg, const double* __restrict__ dfl,
                                const double* __restrict__ amax2, int count, double thr, int relative, double rfac,
                                int64_t nb, double fs, double f_low, double f_high, double df_high,
                                int* __restrict__ m0_out, int* __restrict__ len_out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= count) return;
  const double amp = relative ? thr * rfac * fs * sqrt(amax2[j]) : thr;
  if (!(amp > 0.0)) {
    m0_out[j] = 0;
    len_out[j] = 0;
    return;
  }
  const double fe[4] = {f_low - dfl[j], f_low, f_high, f_high + df_high};
  const double dfe[4] = {dfl[j], dfl[j], df_high, df_high};
  double lo = INFINITY, hi = -INFINITY;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const double c = -((tf2_dphase(tg[j], fe[e]) - tf2_dphase(ref, fe[e])) / kTwoPi);
    const double R = tf2_amp(fe[e]) / tf2_amp(fe[e]);  // B_j / B_ref: one amplitude law
    const double d = cbrt(R / (4.0 * kPi * dfe[e] * dfe[e] * amp));
    lo = fmin(lo, c - d);
    hi = fmax(hi, c + d);
  }
  // a span as long as the grid (a tiny amplitude, or a taper of width 0) keeps the whole
  // grid from lag 0; decided in double, before any integer conversion
  const double flo = floor(lo * fs), fhi = ceil(hi * fs);
  if (!(fhi - flo + 1.0 < (double)nb)) {
    m0_out[j] = 0;
    len_out[j] = (int)nb;
    return;
  }
  const long long m_lo = (long long)flo, m_hi = (long long)fhi;
  long long m0 = m_lo & (nb - 1);
  if (m0 > nb / 2) m0 -= nb;
  m0_out[j] = (int)m0;
  len_out[j] = (int)(m_hi - m_lo + 1);
}

// Real-kernel form: rho -> 2 Re rho in place (imaginary parts zero).
__global__ void k_real_form(double2* __restrict__ rho, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    rho[i] = make_double2(2.0 * rho[i].x, 0.0);
}

__global__ void __launch_bounds__(256) k_ref_phase(Tf2 ref, int64_t nbins, double df, double* __restrict__ psi) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nbins) return;
  psi[k] = (k > 0) ? tf2_phase(ref, (double)k * df) : 0.0;
}

// One row per template (grid.y): K~ over the full length-n buffer.
__global__ void __launch_bounds__(256) k_kernel_spectrum(const Tf2* __restrict__ tg, const double* __restrict__ dfl,
                                                         const double* __restrict__ psi_ref, int64_t n, double df,
                                                         double f_low, double f_high, double df_high,
                                                         double2* __restrict__ K) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int j = blockIdx.y;
  double2 out = make_double2(0.0, 0.0);
  if (k > 0 && k <= n / 2) {
    const double f = (double)k * df;
    const double w = window_w(f, f_low, f_high, dfl[j], df_high);
    if (w > 0.0) {
      const double dpsi = tf2_phase(tg[j], f) - psi_ref[k];
      // K~ = (N_ref / N_j) W conj(h~_j / h~_ref) (Eq. 5 normalised as in Eq. 3).  Every
      // template of the stationary-phase family has the amplitude law A f^-7/6 on the same
      // band, so h~_j / h~_ref = (A_j / A_ref) e^{-i dPsi} and N_j / N_ref = A_j / A_ref: the
      // two amplitude factors cancel exactly for any scales A, and |K~| = W.
      double s, c;
      sincos(dpsi, &s, &c);
      const double a = w / (double)n;
      out = make_double2(a * c, a * s);
    }
  }
  K[(int64_t)j * n + k] = out;
}

__device__ __forceinline__ double mag2_rn(double2 v) { return __dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y)); }

__global__ void __launch_bounds__(1024) k_row_max2(const double2* __restrict__ rho, int64_t n, double* __restrict__ out) {
  const double2* r = rho + (int64_t)blockIdx.x * n;
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, mag2_rn(r[i]));
  __shared__ double sh[1024];
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

struct ArcBest {
  long long gap, m0;
};

__device__ __forceinline__ long long arc_key(long long m, long long n) { return m <= n / 2 ? m : m - n; }

__device__ __forceinline__ void arc_take(ArcBest& b, long long gap, long long m, long long n) {
  if (gap > b.gap || (gap == b.gap && arc_key(m, n) < arc_key(b.m0, n))) {
    b.gap = gap;
    b.m0 = m;
  }
}

// Shortest covering arc of {m : |rho[m]|^2 >= cut2}, one block per template.
// Each thread summarises a contiguous range (first kept, last kept, best internal gap);
// thread 0 joins the summaries in order and closes the circle.
__global__ void __launch_bounds__(1024) k_arc(const double2* __restrict__ rho, int64_t n,
                                              const double* __restrict__ amax2, double thr, int relative,
                                              int* __restrict__ m0_out, int* __restrict__ len_out) {
  const int j = blockIdx.x;
  const double2* r = rho + (int64_t)j * n;
  const double cut2 = __dmul_rn(__dmul_rn(thr, thr), relative ? amax2[j] : 1.0);
  const int nt = blockDim.x;
  const int64_t ch = n / nt;
  const int t = threadIdx.x;
  long long first = -1, last = -1;
  ArcBest b{-1, 0};
  const bool any = relative ? (amax2[j] > 0.0) : true;
  if (any) {
    for (int64_t m = (int64_t)t * ch; m < (int64_t)(t + 1) * ch; ++m) {
      if (mag2_rn(r[m]) >= cut2) {
        if (last >= 0) arc_take(b, m - last - 1, m, n);
        if (first < 0) first = m;
        last = m;
      }
    }
  }
  __shared__ long long s_first[1024], s_last[1024], s_gap[1024], s_m0[1024];
  s_first[t] = first;
  s_last[t] = last;
  s_gap[t] = b.gap;
  s_m0[t] = b.m0;
  __syncthreads();
  if (t == 0) {
    long long gfirst = -1, glast = -1;
    ArcBest g{-1, 0};
    for (int q = 0; q < nt; ++q) {
      if (s_first[q] < 0) continue;
      if (glast >= 0) arc_take(g, s_first[q] - glast - 1, s_first[q], n);
      if (s_gap[q] >= 0) arc_take(g, s_gap[q], s_m0[q], n);
      if (gfirst < 0) gfirst = s_first[q];
      glast = s_last[q];
    }
    if (gfirst < 0) {
      m0_out[j] = 0;
      len_out[j] = 0;
    } else {
      arc_take(g, gfirst + n - glast - 1, gfirst, n);
      m0_out[j] = (int)arc_key(g.m0, n);
      len_out[j] = (int)(n - g.gap);
    }
  }
}

template <typename V>
__global__ void __launch_bounds__(256) k_pack(const double2* __restrict__ rho, int64_t n, const int* __restrict__ m0,
                                              const int* __restrict__ len, const int64_t* __restrict__ off,
                                              V* __restrict__ taps) {
  using R = typename real_of<V>::type;
  const int j = blockIdx.y;
  const int L = len[j];
  const int64_t mask = n - 1;
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < L; l += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = rho[(int64_t)j * n + ((m0[j] + l) & mask)];
    taps[off[j] + l] = cmake<V>((R)v.x, (R)v.y);
  }
}

// Real-kernel form: the real parts only (the imaginary parts are zero after k_real_form).
template <typename R>
__global__ void __launch_bounds__(256) k_pack_real(const double2* __restrict__ rho, int64_t n,
                                                   const int* __restrict__ m0, const int* __restrict__ len,
                                                   const int64_t* __restrict__ off, R* __restrict__ taps) {
  const int j = blockIdx.y;
  const int L = len[j];
  const int64_t mask = n - 1;
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < L; l += (int64_t)gridDim.x * blockDim.x)
    taps[off[j] + l] = (R)rho[(int64_t)j * n + ((m0[j] + l) & mask)].x;
}

}  // namespace

rf_kernels* build_impl(rf_ctx* c, const rf_template& ref, const rf_template* nbrs, int32_t k, const double* inv_psd,
                       double thr, int relative, int64_t n_build, cudaStream_t s) {
  const int64_t n = c->n;
  const bool f64 = c->g.dtype == RF_F64;
  const bool real_form = (relative & RF_KERNEL_REAL) != 0;

  std::unique_ptr<rf_kernels> owner(new rf_kernels());
  rf_kernels* kern = owner.get();
  kern->k = k;
  kern->n = n;
  kern->real = real_form;
  kern->dtype = c->g.dtype;
  const size_t esz = tap_bytes(kern);
  kern->len.assign(k, 0);
  kern->lag0.assign(k, 0);
  kern->offset.assign((size_t)k + 1, 0);
  kern->df_low.assign(k, 0.0);
  kern->grid.assign(k, n);
  if (k == 0) {
    kern->taps.ensure(16);
    kern->len_d.ensure(16);
    kern->lag0_d.ensure(16);
    kern->off_d.ensure(16);
    RF_CUDA(cudaMemsetAsync(kern->off_d.p, 0, sizeof(int64_t), s));
    RF_CUDA(cudaStreamSynchronize(s));
    return owner.release();
  }

  // device scratch: [Tf2 k][dfl k][extent k][Tf2 k, grid order][dfl k, grid order][psi_ref]
  // [amax2][m0][len]
  const int64_t nbins = n / 2 + 1;
  const int64_t kmax_chunk = std::min<int64_t>(k, 4096);
  DevBuf meta;
  const size_t meta_bytes = 2 * sizeof(Tf2) * (size_t)k + sizeof(double) * (3 * (size_t)k + nbins + 8 + kmax_chunk) +
                            2 * sizeof(int) * (size_t)kmax_chunk + 8192;
  meta.ensure(meta_bytes);
  char* mp = static_cast<char*>(meta.p);
  auto carve = [&](size_t bytes) {
    char* r = mp;
    mp += (bytes + 255) & ~(size_t)255;
    return r;
  };
  Tf2* d_tg = reinterpret_cast<Tf2*>(carve(sizeof(Tf2) * k));
  double* d_dfl = reinterpret_cast<double*>(carve(sizeof(double) * k));
  double* d_ext = reinterpret_cast<double*>(carve(sizeof(double) * k));
  Tf2* d_tgs = reinterpret_cast<Tf2*>(carve(sizeof(Tf2) * k));
  double* d_dfls = reinterpret_cast<double*>(carve(sizeof(double) * k));
  double* d_psi = reinterpret_cast<double*>(carve(sizeof(double) * nbins));
  double* d_amax = reinterpret_cast<double*>(carve(sizeof(double) * kmax_chunk));
  int* d_m0 = reinterpret_cast<int*>(carve(sizeof(int) * kmax_chunk));
  int* d_len = reinterpret_cast<int*>(carve(sizeof(int) * kmax_chunk));
  RF_REQUIRE((size_t)(mp - static_cast<char*>(meta.p)) <= meta_bytes, "builder: scratch layout");

  std::vector<Tf2> tg(k);
  for (int j = 0; j < k; ++j) tg[j] = make_tf2(nbrs[j], c->g.pn_order);
  RF_CUDA(cudaMemcpyAsync(d_tg, tg.data(), sizeof(Tf2) * k, cudaMemcpyHostToDevice, s));
  const Tf2 pr = make_tf2(ref, c->g.pn_order);
  k_df_low<<<(k + 127) / 128, 128, 0, s>>>(pr, d_tg, k, c->g.f_low, c->g.df_low_max, d_dfl);
  RF_LAUNCHED();
  RF_CUDA(cudaMemcpyAsync(kern->df_low.data(), d_dfl, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  // build grid per neighbour
  if (n_build < 0) {
    std::vector<double> ext(k);
    k_grid_extent<<<(k + 127) / 128, 128, 0, s>>>(pr, d_tg, d_dfl, k, c->g.fs, c->g.f_low, c->g.f_high, c->g.df_high,
                                                  d_ext);
    RF_LAUNCHED();
    RF_CUDA(cudaMemcpyAsync(ext.data(), d_ext, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
    RF_CUDA(cudaStreamSynchronize(s));
    for (int j = 0; j < k; ++j) {
      int64_t nb = 16;
      while ((double)nb < 4.0 * ext[j] && nb < n) nb *= 2;
      kern->grid[j] = std::min<int64_t>(nb, n);
    }
  } else if (n_build > 0) {
    for (int j = 0; j < k; ++j) kern->grid[j] = n_build;
  }
  RF_CUDA(cudaStreamSynchronize(s));  // df_low is on the host
  // neighbours in grid order (stable), chunks of one grid
  std::vector<int> order(k);
  for (int j = 0; j < k; ++j) order[j] = j;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return kern->grid[a] < kern->grid[b]; });
  {
    std::vector<Tf2> tgs(k);
    std::vector<double> dfls(k);
    for (int q = 0; q < k; ++q) {
      tgs[q] = tg[order[q]];
      dfls[q] = kern->df_low[order[q]];
    }
    RF_CUDA(cudaMemcpyAsync(d_tgs, tgs.data(), sizeof(Tf2) * k, cudaMemcpyHostToDevice, s));
    RF_CUDA(cudaMemcpyAsync(d_dfls, dfls.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s));
    RF_CUDA(cudaStreamSynchronize(s));  // the host vectors go out of scope
  }

  // per kernel: its taps in a part buffer (one per chunk) and its place there
  std::vector<std::unique_ptr<DevBuf>> parts;
  std::vector<int> part_of(k);
  std::vector<int64_t> at_in_part(k);
  std::vector<int> hm0(kmax_chunk), hlen(kmax_chunk);
  DevBuf rows;
  int64_t psi_grid = 0;
  for (int q0 = 0; q0 < k;) {
    const int64_t nb = kern->grid[order[q0]];
    // templates per chunk: three complex128 rows of nb per template, about 1.5 GB in total
    const int64_t per = 3 * nb * (int64_t)sizeof(double2);
    int64_t chunk = std::max<int64_t>(1, ((int64_t)1536 << 20) / per);
    chunk = std::min<int64_t>(chunk, kmax_chunk);
    int cnt = 0;
    while (q0 + cnt < k && cnt < chunk && kern->grid[order[q0 + cnt]] == nb) ++cnt;
    const double dfb = c->g.fs / (double)nb;
    if (psi_grid != nb) {
      k_ref_phase<<<(unsigned)((nb / 2 + 1 + 255) / 256), 256, 0, s>>>(pr, nb / 2 + 1, dfb, d_psi);
      RF_LAUNCHED();
      psi_grid = nb;
    }
    rows.ensure((size_t)3 * cnt * nb * sizeof(double2));
    double2* bufK = rows.as<double2>();
    double2* bufR = bufK + cnt * nb;
    double2* bufT = bufR + cnt * nb;
    dim3 g1((unsigned)((nb + 255) / 256), (unsigned)cnt);
    k_kernel_spectrum<<<g1, 256, 0, s>>>(d_tgs + q0, d_dfls + q0, d_psi, nb, dfb, c->g.f_low,
                                         c->g.f_high, c->g.df_high, bufK);
    RF_LAUNCHED();
    fft_c2c_f64(bufK, bufR, bufT, nb, cnt, +1, c->tw64.as<double2>(), n, s);
    if (relative & RF_KERNEL_REAL) {
      k_real_form<<<(unsigned)std::min<int64_t>(4096, (cnt * nb + 255) / 256), 256, 0, s>>>(bufR, cnt * nb);
      RF_LAUNCHED();
    }
    k_row_max2<<<cnt, 1024, 0, s>>>(bufR, nb, d_amax);
    RF_LAUNCHED();
    if (relative & RF_TRUNC_ANALYTIC) {
      k_analytic_span<<<(cnt + 63) / 64, 64, 0, s>>>(pr, d_tgs + q0, d_dfls + q0, d_amax, cnt, thr,
                                                     relative & RF_TRUNC_RELATIVE,
                                                     (relative & RF_KERNEL_REAL) ? 1.0 : 2.0, nb, c->g.fs,
                                                     c->g.f_low, c->g.f_high, c->g.df_high, d_m0, d_len);
    } else {
      const int nt = (int)std::min<int64_t>(1024, nb);
      k_arc<<<cnt, nt, 0, s>>>(bufR, nb, d_amax, thr, relative & RF_TRUNC_RELATIVE, d_m0, d_len);
    }
    RF_LAUNCHED();
    RF_CUDA(cudaMemcpyAsync(hm0.data(), d_m0, sizeof(int) * cnt, cudaMemcpyDeviceToHost, s));
    RF_CUDA(cudaMemcpyAsync(hlen.data(), d_len, sizeof(int) * cnt, cudaMemcpyDeviceToHost, s));
    RF_CUDA(cudaStreamSynchronize(s));
    std::vector<int64_t> off(cnt + 1, 0);
    for (int q = 0; q < cnt; ++q) {
      const int j = order[q0 + q];
      kern->lag0[j] = hm0[q];
      kern->len[j] = hlen[q];
      part_of[j] = (int)parts.size();
      at_in_part[j] = off[q];
      off[q + 1] = off[q] + hlen[q];
    }
    std::unique_ptr<DevBuf> part(new DevBuf());
    part->ensure(std::max<size_t>(16, (size_t)off[cnt] * esz));
    DevBuf offd;
    offd.ensure(sizeof(int64_t) * (cnt + 1));
    RF_CUDA(cudaMemcpyAsync(offd.p, off.data(), sizeof(int64_t) * (cnt + 1), cudaMemcpyHostToDevice, s));
    dim3 g2(64, (unsigned)cnt);
    if (real_form && f64)
      k_pack_real<double><<<g2, 256, 0, s>>>(bufR, nb, d_m0, d_len, offd.as<int64_t>(), part->as<double>());
    else if (real_form)
      k_pack_real<float><<<g2, 256, 0, s>>>(bufR, nb, d_m0, d_len, offd.as<int64_t>(), part->as<float>());
    else if (f64)
      k_pack<double2><<<g2, 256, 0, s>>>(bufR, nb, d_m0, d_len, offd.as<int64_t>(), part->as<double2>());
    else
      k_pack<float2><<<g2, 256, 0, s>>>(bufR, nb, d_m0, d_len, offd.as<int64_t>(), part->as<float2>());
    RF_LAUNCHED();
    RF_CUDA(cudaStreamSynchronize(s));  // offd and the rows are reused
    parts.push_back(std::move(part));
    q0 += cnt;
  }
  for (int j = 0; j < k; ++j) kern->offset[j + 1] = kern->offset[j] + kern->len[j];
  const int64_t total = kern->offset[k];
  kern->taps.ensure(std::max<size_t>(16, (size_t)total * esz));
  // taps in neighbour order: one copy per part when the order is unchanged, else one per kernel
  bool identity = true;
  for (int q = 0; q < k && identity; ++q) identity = order[q] == q;
  if (identity) {
    int64_t at = 0;
    for (size_t pi = 0; pi < parts.size(); ++pi) {
      int64_t elems = 0;
      for (int j = 0; j < k; ++j)
        if (part_of[j] == (int)pi) elems += kern->len[j];
      if (elems)
        RF_CUDA(cudaMemcpyAsync(static_cast<char*>(kern->taps.p) + at * esz, parts[pi]->p, elems * esz,
                                cudaMemcpyDeviceToDevice, s));
      at += elems;
    }
  } else {
    for (int j = 0; j < k; ++j)
      if (kern->len[j])
        RF_CUDA(cudaMemcpyAsync(static_cast<char*>(kern->taps.p) + kern->offset[j] * esz,
                                static_cast<char*>(parts[part_of[j]]->p) + at_in_part[j] * esz,
                                (size_t)kern->len[j] * esz, cudaMemcpyDeviceToDevice, s));
  }
  kern->max_len = *std::max_element(kern->len.begin(), kern->len.end());
  kern->len_d.ensure(sizeof(int32_t) * k);
  kern->lag0_d.ensure(sizeof(int32_t) * k);
  kern->off_d.ensure(sizeof(int64_t) * (k + 1));
  RF_CUDA(cudaMemcpyAsync(kern->len_d.p, kern->len.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, s));
  RF_CUDA(cudaMemcpyAsync(kern->lag0_d.p, kern->lag0.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, s));
  RF_CUDA(cudaMemcpyAsync(kern->off_d.p, kern->offset.data(), sizeof(int64_t) * (k + 1), cudaMemcpyHostToDevice, s));
  RF_CUDA(cudaStreamSynchronize(s));
  return owner.release();
}

rf_kernels* import_impl(rf_ctx* c, int32_t k, const int32_t* lag0, const int32_t* len, const void* taps, bool real) {
  std::unique_ptr<rf_kernels> owner(new rf_kernels());
  rf_kernels* kern = owner.get();
  kern->k = k;
  kern->n = c->n;
  kern->dtype = c->g.dtype;
  kern->real = real;
  const size_t esz = tap_bytes(kern);
  kern->grid.assign(k, c->n);
  kern->len.assign(len, len + k);
  kern->lag0.assign(lag0, lag0 + k);
  kern->offset.assign((size_t)k + 1, 0);
  kern->df_low.assign(k, std::nan(""));
  for (int j = 0; j < k; ++j) kern->offset[j + 1] = kern->offset[j] + len[j];
  kern->max_len = k ? *std::max_element(kern->len.begin(), kern->len.end()) : 0;
  const int64_t total = kern->offset[k];
  kern->taps.ensure(std::max<size_t>(16, (size_t)total * esz));
  kern->len_d.ensure(std::max<size_t>(16, sizeof(int32_t) * k));
  kern->lag0_d.ensure(std::max<size_t>(16, sizeof(int32_t) * k));
  kern->off_d.ensure(sizeof(int64_t) * (k + 1));
  if (total) RF_CUDA(cudaMemcpy(kern->taps.p, taps, (size_t)total * esz, cudaMemcpyHostToDevice));
  if (k) {
    RF_CUDA(cudaMemcpy(kern->len_d.p, len, sizeof(int32_t) * k, cudaMemcpyHostToDevice));
    RF_CUDA(cudaMemcpy(kern->lag0_d.p, lag0, sizeof(int32_t) * k, cudaMemcpyHostToDevice));
  }
  RF_CUDA(cudaMemcpy(kern->off_d.p, kern->offset.data(), sizeof(int64_t) * (k + 1), cudaMemcpyHostToDevice));
  return owner.release();
}

}  // namespace rf
