// Four-step FP32 FFT of n = N1 N2 points in two passes through HBM (the matched filter of
// Eq. 2 at large n: the data transform and the per-template inverse transforms).
//
// With the input index j = N2 a + b (a < N1, b < N2) and the output index k = k1 + N1 k2,
//   X[k1 + N1 k2] = sum_b w_N2^(b k2) [ w_n^(b k1) sum_a x[N2 a + b] w_N1^(a k1) ],
// w_m = exp(sign 2 pi i / m).  Pass 1 transforms the N2 columns (N1 points each, stride N2),
// multiplies by w_n^(b k1) and stores the result in the same layout; pass 2 transforms the
// N1 rows (N2 contiguous points) and stores X[k1 + N1 k2] (natural order, a transposed store).
//
// Both passes run the shared-memory block FFT (blockfft.cuh) on several lines per thread
// block: pass 1 on G adjacent columns, whose lanes interleave so that every load and store of
// a warp covers runs of G consecutive elements; pass 2 on R adjacent rows, staged through
// shared memory for the transposed store (runs of R elements).  Lines of a tile start at
// offsets 16/G float2 apart modulo 16 bank pairs, which keeps the half-warp accesses of every
// stage conflict free.
//
// The twiddle w_n^m (m = b k1 < n) is the product of two table entries: w_n^(m mod 2^s) and
// w_n^(2^s floor(m / 2^s)), with 2^s = 2^ceil(log2(n) / 2); the tables (about 2 sqrt(n)
// entries) stay in cache.
//
// Modes of pass 1: real input (the data transform), complex input, and the one-sided product
// X[k] F[k] for k <= n/2, zero above (the matched-filter integrand, formed on load).
#include "blockfft.cuh"
#include "rf_internal.h"

namespace rf {

namespace {

constexpr int kF4Real = 0;
constexpr int kF4Complex = 1;
constexpr int kF4Product = 2;

// float2 entries of one line's shared-memory region in a tile of G lines.
template <int L, int G>
__host__ __device__ constexpr int f4_line() {
  return L + L / 16 + 16 / G;
}

template <int L, int G>
constexpr size_t f4_smem() {
  return sizeof(float2) * (size_t)G * (size_t)f4_line<L, G>();
}

// Pass 1: columns col0 .. col0 + G - 1 of batch row blockIdx.y; L = N1.
template <int L, int G, int MODE, int SIGN>
__global__ void __launch_bounds__(G * L / 16) k_fft4_cols(const void* __restrict__ in, const float2* __restrict__ F,
                                                          int64_t fstride, float2* __restrict__ out, int n2log,
                                                          const float2* __restrict__ twb,
                                                          const float2* __restrict__ tw4, int lo_bits) {
  using S = BlockFFTShape<L>;
  constexpr int NT = S::NT;
  constexpr int RL = S::RL;
  extern __shared__ float2 f4_sm[];
  const int c = (int)threadIdx.x % G;
  const int ltid = (int)threadIdx.x / G;
  const int64_t N2 = (int64_t)1 << n2log;
  const int64_t n = N2 * L;
  const int64_t col = (int64_t)blockIdx.x * G + c;
  const int64_t boff = (int64_t)blockIdx.y * n;
  // element (a = ltid + t NT, col) sits at j0 + t NT N2
  const int64_t j0 = (int64_t)ltid * N2 + col;
  const int64_t tstep = (int64_t)NT * N2;
  float2 v[16];
  if constexpr (MODE == kF4Real) {
    const float* p = static_cast<const float*>(in) + boff + j0;
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t] = make_float2(p[t * tstep], 0.f);
  } else if constexpr (MODE == kF4Complex) {
    const float2* p = static_cast<const float2*>(in) + boff + j0;
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t] = p[t * tstep];
  } else {
    // X is one spectrum shared by the batch; F holds one filter of n/2 + 1 values per row.
    // Rows a > N1/2 lie above n/2 (zero); row N1/2 holds only column 0.
    const float2* px = static_cast<const float2*>(in) + j0;
    const float2* pf = F + (int64_t)blockIdx.y * fstride + j0;
    const int64_t lim = n / 2 - j0;
#pragma unroll
    for (int t = 0; t < 16; ++t)
      v[t] = t * tstep <= lim ? cmul(px[t * tstep], pf[t * tstep]) : make_float2(0.f, 0.f);
  }
  block_fft<L, SIGN>(v, f4_sm + c * f4_line<L, G>(), twb, ltid);
  // v[q RL + t] holds the column's bin k1 = ltid + NT u, u = q + t 16/RL (every u < 16 once).
  // Twiddle w_n^(col k1) = w_n^(col ltid) e^u with e = w_n^(col NT): e, e^2, e^4 and e^8 come
  // from the tables (a product of two entries each, m = col NT 2^i < n), e^3, e^5 .. e^7 by at
  // most two more products, and e^(u + 8) = e^u e^8 (a few ulp in all).
  const unsigned lomask = (1u << lo_bits) - 1u;
  const float2* thi = tw4 + (1u << lo_bits);
  const auto table = [&](unsigned m) { return cmul(__ldg(tw4 + (m & lomask)), __ldg(thi + (m >> lo_bits))); };
  const unsigned cu = (unsigned)col;  // col k1 < n <= 2^24
  const float2 b0 = table(cu * (unsigned)ltid);
  const float2 e1 = table(cu * NT), e2 = table(cu * 2u * NT), e4 = table(cu * 4u * NT), e8 = table(cu * 8u * NT);
  float2* o = out + boff + j0;  // bin k1 goes to row k1: o + NT u N2
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    float2 eu;
    if (u == 0) eu = make_float2(1.f, 0.f);
    else if (u == 1) eu = e1;
    else if (u == 2) eu = e2;
    else if (u == 3) eu = cmul(e2, e1);
    else if (u == 4) eu = e4;
    else if (u == 5) eu = cmul(e4, e1);
    else if (u == 6) eu = cmul(e4, e2);
    else eu = cmul(e4, cmul(e2, e1));
    const float2 w = u == 0 ? b0 : cmul(b0, eu);
    const float2 w8 = cmul(w, e8);
    constexpr int QN = 16 / RL;
    const int r0 = (u % QN) * RL + u / QN;              // register of bin ltid + NT u
    const int r8 = ((u + 8) % QN) * RL + (u + 8) / QN;  // register of bin ltid + NT (u + 8)
    o[(int64_t)(u * NT) * N2] = tw_apply<SIGN>(v[r0], w);
    o[(int64_t)((u + 8) * NT) * N2] = tw_apply<SIGN>(v[r8], w8);
  }
}

// Pass 2: rows row0 .. row0 + R - 1 of batch row blockIdx.y; L = N2.  Output k1 + N1 k2.
template <int L, int R, int SIGN>
__global__ void __launch_bounds__(R * L / 16) k_fft4_rows(const float2* __restrict__ in, float2* __restrict__ out,
                                                          int n1log, const float2* __restrict__ twb) {
  using S = BlockFFTShape<L>;
  constexpr int NT = S::NT;
  constexpr int RL = S::RL;
  constexpr int SL = f4_line<L, R>();
  extern __shared__ float2 f4_sm[];
  const int g = (int)threadIdx.x / NT;
  const int ltid = (int)threadIdx.x % NT;
  const int64_t N1 = (int64_t)1 << n1log;
  const int64_t n = N1 * L;
  const int64_t row0 = (int64_t)blockIdx.x * R;
  const float2* src = in + (int64_t)blockIdx.y * n + (row0 + g) * L;
  float2 v[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) v[t] = src[ltid + t * NT];
  float2* sm = f4_sm + g * SL;
  block_fft<L, SIGN>(v, sm, twb, ltid);
  __syncthreads();  // the last stage has read its inputs from shared memory
#pragma unroll
  for (int q = 0; q < 16 / RL; ++q)
#pragma unroll
    for (int t = 0; t < RL; ++t) sm[ltid + q * NT + t * (L / RL)] = v[q * RL + t];
  __syncthreads();
  float2* dst = out + (int64_t)blockIdx.y * n + row0;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int f = (int)threadIdx.x + i * (R * NT);
    const int gg = f % R;
    const int k2 = f / R;
    dst[gg + (int64_t)k2 * N1] = f4_sm[gg * SL + k2];
  }
}

constexpr int kF4MinLog = 18;  // N1, N2 >= 512: the block FFT tables start at 2^9
constexpr int kF4MaxLog = 24;  // N1, N2 <= 4096

// Tile widths: G columns of N1 points (G N1 / 16 <= 1024 threads), R rows of N2 points.
template <int L> constexpr int f4_cols_g() { return L >= 4096 ? 4 : 8; }
template <int L> constexpr int f4_rows_r() { return 4; }

template <int L, int MODE, int SIGN>
void launch_cols(const void* in, const float2* F, int64_t fstride, float2* out, int n2log, int batch,
                 const rf_ctx* c, cudaStream_t s) {
  constexpr int G = f4_cols_g<L>();
  const auto fn = k_fft4_cols<L, G, MODE, SIGN>;
  constexpr size_t smem = f4_smem<L, G>();
  RF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int lb = BlockFFTShape<L>::LOGB;
  dim3 grid((unsigned)(((int64_t)1 << n2log) / G), (unsigned)batch);
  fn<<<grid, G * L / 16, smem, s>>>(in, F, fstride, out, n2log, c->twb32.as<float2>() + c->twb_off[lb],
                                     c->tw4.as<float2>(), c->tw4_lo_bits);
  RF_LAUNCHED();
}

template <int L, int SIGN>
void launch_rows(const float2* in, float2* out, int n1log, int batch, const rf_ctx* c, cudaStream_t s) {
  constexpr int R = f4_rows_r<L>();
  const auto fn = k_fft4_rows<L, R, SIGN>;
  constexpr size_t smem = f4_smem<L, R>();
  RF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int lb = BlockFFTShape<L>::LOGB;
  dim3 grid((unsigned)(((int64_t)1 << n1log) / R), (unsigned)batch);
  fn<<<grid, R * L / 16, smem, s>>>(in, out, n1log, c->twb32.as<float2>() + c->twb_off[lb]);
  RF_LAUNCHED();
}

int ilog2(int64_t n) {
  int b = 0;
  while (((int64_t)1 << b) < n) ++b;
  return b;
}

template <int MODE, int SIGN>
void cols_dispatch(int n1log, const void* in, const float2* F, int64_t fstride, float2* out, int n2log, int batch,
                   const rf_ctx* c, cudaStream_t s) {
  switch (n1log) {
    case 9: launch_cols<512, MODE, SIGN>(in, F, fstride, out, n2log, batch, c, s); break;
    case 10: launch_cols<1024, MODE, SIGN>(in, F, fstride, out, n2log, batch, c, s); break;
    case 11: launch_cols<2048, MODE, SIGN>(in, F, fstride, out, n2log, batch, c, s); break;
    default: launch_cols<4096, MODE, SIGN>(in, F, fstride, out, n2log, batch, c, s); break;
  }
}

template <int SIGN>
void rows_dispatch(int n2log, const float2* in, float2* out, int n1log, int batch, const rf_ctx* c,
                   cudaStream_t s) {
  switch (n2log) {
    case 9: launch_rows<512, SIGN>(in, out, n1log, batch, c, s); break;
    case 10: launch_rows<1024, SIGN>(in, out, n1log, batch, c, s); break;
    case 11: launch_rows<2048, SIGN>(in, out, n1log, batch, c, s); break;
    default: launch_rows<4096, SIGN>(in, out, n1log, batch, c, s); break;
  }
}

// N1 = 2^floor(log2(n) / 2) points per column, N2 = n / N1 per row
void split(int64_t n, int& n1log, int& n2log) {
  const int b = ilog2(n);
  n1log = b / 2;
  n2log = b - n1log;
}

void check(const rf_ctx* c, const void* in, const void* out, const void* tmp, int batch) {
  RF_REQUIRE(fft4_supported(c->n), "fft4: n=%lld is outside 2^%d .. 2^%d", (long long)c->n, kF4MinLog, kF4MaxLog);
  RF_REQUIRE(c->tw4.p != nullptr, "fft4: twiddle tables missing");
  RF_REQUIRE(batch >= 1 && batch <= 65535, "fft4: batch %d out of range", batch);
  RF_REQUIRE(in != out && in != tmp && out != tmp, "fft4: buffers must be distinct");
}

}  // namespace

bool fft4_supported(int64_t n) {
  if (n <= 0 || (n & (n - 1)) != 0) return false;
  const int b = ilog2(n);
  return b >= kF4MinLog && b <= kF4MaxLog;
}

int fft4_lo_bits(int64_t n) { return (ilog2(n) + 1) / 2; }

void fft4_forward_real(const rf_ctx* c, const float* x, float2* out, float2* tmp, cudaStream_t s) {
  check(c, x, out, tmp, 1);
  int n1log, n2log;
  split(c->n, n1log, n2log);
  cols_dispatch<kF4Real, -1>(n1log, x, nullptr, 0, tmp, n2log, 1, c, s);
  rows_dispatch<-1>(n2log, tmp, out, n1log, 1, c, s);
}

void fft4_inverse(const rf_ctx* c, const float2* in, float2* out, float2* tmp, int batch, cudaStream_t s) {
  check(c, in, out, tmp, batch);
  int n1log, n2log;
  split(c->n, n1log, n2log);
  cols_dispatch<kF4Complex, +1>(n1log, in, nullptr, 0, tmp, n2log, batch, c, s);
  rows_dispatch<+1>(n2log, tmp, out, n1log, batch, c, s);
}

void fft4_inverse_product(const rf_ctx* c, const float2* X, const float2* F, int64_t fstride, float2* out,
                          float2* tmp, int batch, cudaStream_t s) {
  check(c, X, out, tmp, batch);
  RF_REQUIRE(fstride >= c->n / 2 + 1, "fft4: filter stride %lld below n/2 + 1", (long long)fstride);
  int n1log, n2log;
  split(c->n, n1log, n2log);
  cols_dispatch<kF4Product, +1>(n1log, X, F, fstride, tmp, n2log, batch, c, s);
  rows_dispatch<+1>(n2log, tmp, out, n1log, batch, c, s);
}

}  // namespace rf
