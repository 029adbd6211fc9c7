// Internal declarations shared by the translation units of librf.so.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <memory>
#include <string>
#include <vector>

#include "rf.h"

namespace rf {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
void clear_error();

struct Fail {
  rf_status st;
};

#define RF_CUDA(expr)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (expr);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      ::rf::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                      __LINE__);                                                       \
      throw ::rf::Fail{RF_ECUDA};                                                      \
    }                                                                                  \
  } while (0)

#define RF_REQUIRE(cond, ...)        \
  do {                               \
    if (!(cond)) {                   \
      ::rf::set_error(__VA_ARGS__);  \
      throw ::rf::Fail{RF_EINVAL};   \
    }                                \
  } while (0)

// Launch check: catches configuration errors of the launch just made, and counts it.
void count_launch();
#define RF_LAUNCHED()                    \
  do {                                   \
    RF_CUDA(cudaGetLastError());         \
    ::rf::count_launch();                \
  } while (0)

// ---------------------------------------------------------------- device buffers
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  // Grow to at least `b` bytes (contents are not kept).
  void ensure(size_t b);
  template <typename T>
  T* as() const { return static_cast<T*>(p); }
};

// Pinned host memory, grown on demand (contents are not kept).
struct PinBuf {
  void* p = nullptr;
  size_t bytes = 0;
  PinBuf() = default;
  PinBuf(const PinBuf&) = delete;
  PinBuf& operator=(const PinBuf&) = delete;
  ~PinBuf() {
    if (p) cudaFreeHost(p);
  }
  void ensure(size_t b) {
    if (b <= bytes) return;
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
    RF_CUDA(cudaMallocHost(&p, b));
    bytes = b;
  }
};

// Work item of the batched and two-phase overlap-save launches: one neighbour's partition
// spectra C (P of them), the segment spectra Zs of its reference, its first lag and its row.
struct OsItem {
  const float2* C;
  const float2* Zs;
  int P;
  int lag0;
  long long row;
};
// Two-phase overlap-save (reconstruct_bins.cu): items sorted by partition count, cut into waves
// of (item tile, time tile); phase 1 per-bin partition sums into a buffer, phase 2 block tails.
struct BinsWave {
  int item0, nitems;  // items [item0, item0 + nitems) of the plan
  int s0, ns;         // output blocks [s0, s0 + ns)
  int pmax;           // most partitions among the tile's items
};
struct BinsPlan {
  int B = 0, Lp = 0, NQ = 0, NB = 0;
  bool herm = false;
  std::vector<OsItem> items;  // in plan order
  std::vector<BinsWave> waves;
  size_t y_bytes = 0;         // buffers of two waves' partition sums (waves alternate)
  size_t y_stride = 0;        // float2 elements from the first wave buffer to the second
};

// ---------------------------------------------------------------- template model
// TaylorF2 coefficients of one template (App. A, Eq. A1), prepared on the host
// from the published post-Newtonian series and evaluated on the device in FP64.
struct Tf2 {
  double M;        // total mass in seconds
  double eta;
  double tc, phic;
  double pref;     // 3 / (128 eta)
  double a[8];     // constant parts of alpha_0..alpha_7
  double a5log;    // coefficient of ln(v / v_lso) (v^0 term)
  double a6log;    // coefficient of v ln(4 v)
};
Tf2 make_tf2(const rf_template& t, int pn_order);
// streaming over data longer than one segment (stream.cu)
void stream_winmax_impl(rf_ctx* c, const void* x_host, int64_t total, int32_t G, const void* filt,
                        rf_kernels* const* ks, int64_t W, int64_t guard, float* ref_max, int64_t* ref_arg,
                        float* nbr_max, int64_t* nbr_arg, cudaStream_t s);
// template-bank structuring on the host (bank.cu)
void bank_structure_impl(const rf_template* bank, int32_t count, double f_low, int pn_order, double max_spread,
                         int32_t max_size, int32_t* set_of, int32_t* ref_of_set, int32_t* n_sets,
                         double* duration_out);

}  // namespace rf

// ---------------------------------------------------------------- opaque handles
struct rf_ctx {
  rf_grid g{};
  int device = 0;
  int64_t n = 0;
  int nsm = 0;
  // Twiddle tables w[m] = exp(-2 pi i m / n), m < n: FP64 and FP32 copies.
  rf::DevBuf tw64, tw32;
  // Stage twiddle tables of the block FFTs (float2), B = 2^9 .. 2^14; the tables of
  // block size 2^b start at entry twb_off[b].
  rf::DevBuf twb32;
  int64_t twb_off[16] = {0};
  // Four-step FFT twiddles (float2): w[m] = exp(-2 pi i m / n) for m < 2^tw4_lo_bits, then
  // w[2^tw4_lo_bits m] for m < n / 2^tw4_lo_bits; empty where the four-step FFT does not apply.
  rf::DevBuf tw4;
  int tw4_lo_bits = 0;
  // Workspaces (grid dtype complex unless stated).
  rf::DevBuf xf;       // data spectrum, complex[n]
  rf::DevBuf fa, fb;   // FFT ping-pong, complex[n]
  rf::DevBuf red;      // FP64 reduction scratch
  rf::DevBuf scratch;  // growable: packed window keys, OS block spectra, builder chunks
  rf::DevBuf scratch2;
  rf::DevBuf mf_tmp;   // inverse-transform temporaries of the stored-filter matched filter
  rf::DevBuf status;   // int: device-side error status (RF_ETIMEOUT from bounded waits), 0 if none
  size_t reserved = 0;
  int64_t max_chunk = 0;  // builder templates per chunk
  // Batched overlap-save plan (rf_reconstruct_batched): work items, reference pointers,
  // segment spectra of every reference and packed window keys, kept while the same
  // references and kernel sets come back (so repeated calls allocate and copy nothing).
  std::vector<unsigned long long> batch_key;
  std::vector<int64_t> batch_lay_off;  // work items of layout bucket b: [off[b], off[b+1])
  int64_t batch_rows = 0, batch_nw = 0;
  rf::DevBuf batch_items, batch_zptr, batch_zs, batch_keys;
  // work units (item * nchunk + chunk) in launch order, bucket after bucket: per reference, tiles
  // of output chunks x neighbours small enough that their segment and partition spectra stay
  // in L2 while the units of a tile run
  rf::DevBuf batch_order;
  rf::DevBuf mix_tmp;  // rows of buckets that run the direct or tensor-core form, before scattering
  rf::DevBuf bins_y;   // two-phase overlap-save: one wave's partition sums
  rf::DevBuf bins_e0;  // two-phase 32768-point tail: one 16384-point half transform per SM
  // Two-phase waves run phase 2 on this side stream, so that phase 1 of the next wave (on the
  // caller's stream, into the other buffer) can fill SMs that phase 2 leaves idle.  Events:
  // fork, join, phase 1 done (two buffers), phase 2 done (two buffers).
  cudaStream_t bins_side = nullptr;
  cudaEvent_t bins_ev[6] = {};
  rf_ctx() = default;
  rf_ctx(const rf_ctx&) = delete;
  rf_ctx& operator=(const rf_ctx&) = delete;
  ~rf_ctx();
  std::vector<std::shared_ptr<rf::BinsPlan>> batch_bins;  // per bucket (null unless two-phase)
  rf::DevBuf batch_bins_items;                            // their items, bucket after bucket
  std::vector<int64_t> batch_bins_off;
  std::vector<int64_t> batch_unit_off;  // units of layout bucket b: [off[b], off[b+1])
  std::vector<int> batch_sc;            // output blocks per unit, per bucket
  // Streaming (rf_stream_winmax): two device strain buffers, the references' series, the window
  // peaks, and one pinned host block for the strain staging and the peaks; kept between calls.
  rf::DevBuf st_x[2], st_z, st_pm, st_pa;
  rf::PinBuf st_pin;
};


// One layout bucket of a kernel set: the neighbours whose lengths fall in [cut_lo, next
// bucket's cut_lo) run overlap-save with block size B and partitions of Lp taps (single-pass,
// or RF_ALGO_OS_BINS: two-phase, partition sums per bin), or (algo RF_ALGO_GEMM /
// RF_ALGO_DIRECT) the tensor-core or CUDA-core direct sum on `sub`, a kernel set holding just
// those neighbours, whose rows are then scattered to their places.
struct OsBucket {
  int32_t cut_lo = 0;
  int B = 0, Lp = 0;
  int algo = 2;              // RF_ALGO_OS
  int prec = 0;              // split precision of a tensor-core bucket
  int gemm_nj = 0, gemm_s = 0;  // its tile layout (0, 0: the library's rule)
  std::vector<int32_t> idx;  // neighbour indices, increasing
  rf::DevBuf idx_d;          // int32 copy of idx
  std::shared_ptr<rf_kernels> sub;
  std::shared_ptr<rf::BinsPlan> bins;  // two-phase plan of this bucket alone (single-reference calls)
  rf::DevBuf bins_items_d;             // its items on the device
};

struct rf_kernels {
  int32_t k = 0;
  int64_t n = 0;
  int32_t dtype = 0;
  std::vector<int32_t> len, lag0;
  std::vector<int64_t> offset;
  std::vector<double> df_low;
  std::vector<int64_t> grid;   // build grid of each kernel (its lags are signed on it)
  int32_t max_len = 0;
  // Real-kernel form (the paper's r = 2 Re of the App. A integrand): taps stored as real values
  // of the grid dtype (half the bytes), complex x real products in the direct form, Hermitian
  // half spectra (bins 0..B/2) in the overlap-save preparation.
  bool real = false;
  rf::DevBuf taps;             // packed taps (grid dtype complex, or grid dtype real when `real`)
  rf::DevBuf len_d, lag0_d;    // int32[k]
  rf::DevBuf off_d;            // int64[k+1]
  // Overlap-save preparation (FP32 only): one or more layout buckets by kernel length; kernel j
  // of a bucket with (B, Lp) has P_j = ceil(L_j / Lp) partition spectra FFT_B(taps) / B,
  // stored bucket after bucket.
  bool os_ready = false;
  int os_B = 0;                       // layout of the first bucket
  int os_Lp = 0;                      // partition length (B/2, B/4 or B/8)
  std::vector<OsBucket> os_buckets;
  unsigned long long os_version = 0;  // changes whenever the spectra are rebuilt
  std::vector<int32_t> os_parts;
  std::vector<int64_t> os_off;
  rf::DevBuf os_spec;      // float2, sum_j P_j B_j values
  rf::DevBuf os_off_d;     // int64 [k]: element offset of kernel j's first partition spectrum
  rf::DevBuf os_parts_d;   // int32 [k]
  // Tensor-core direct form: split-BF16 (or TF32) tap operands per group of gemm_NJ neighbours and
  // gemm_S output shifts, taps padded to gemm_LP and extended to gemm_NCK chunks of gemm_KC
  // (see reconstruct_gemm.cu).
  // Form chosen by rf_autotune (RF_ALGO_AUTO then follows it; 0 when not tuned).
  int tuned_algo = 0, tuned_prec = 0;
  bool gemm_ready = false;
  int gemm_prec = 0, gemm_terms = 0, gemm_KC = 0, gemm_NCK = 0, gemm_NJ = 0, gemm_S = 1, gemm_LP = 0;
  bool gemm_tf32 = false;
  int gemm_pref_nj = 0, gemm_pref_s = 0;  // requested tile layout (0, 0: the rule)
  rf::DevBuf gemm_B;
};

namespace rf {

// Bytes of one packed tap of a kernel set: a complex or (real form) a real value of the grid dtype.
inline size_t tap_bytes(const rf_kernels* k) {
  const size_t r = k->dtype == RF_F64 ? sizeof(double) : sizeof(float);
  return k->real ? r : 2 * r;
}

// ---------------------------------------------------------------- FFT (fft.cu)
// Batched out-of-place Stockham FFT of length n (power of two) over `batch`
// contiguous rows.  sign -1: forward, +1: inverse (unnormalised).  Uses `tmp`
// (same size as in/out) as the ping-pong buffer.  in, out, tmp must be distinct.
void fft_c2c_f64(const double2* in, double2* out, double2* tmp, int64_t n, int batch, int sign,
                 const double2* tw_table, int64_t table_n, cudaStream_t s);
// Inverse transform (unnormalised) of the one-sided product X[k] F_b[k] (k <= n/2, zero
// above) for `batch` filters F_b = F + b fstride; the product is formed in the first pass.
void ifft_product_f64(const double2* X, const double2* F, int64_t fstride, double2* out, double2* tmp, int64_t n,
                      int batch, const double2* tw, int64_t table_n, cudaStream_t s);
void ifft_product_f32(const float2* X, const float2* F, int64_t fstride, float2* out, float2* tmp, int64_t n,
                      int batch, const float2* tw, int64_t table_n, cudaStream_t s);
void fft_c2c_f32(const float2* in, float2* out, float2* tmp, int64_t n, int batch, int sign,
                 const float2* tw_table, int64_t table_n, cudaStream_t s);
// Four-step FP32 transforms of the context's n (fft4.cu), for n = 2^18 .. 2^24: two passes
// through HBM.  Forward of real data (natural order out), the unnormalised inverse of batch
// complex rows, and the inverse of the one-sided product X[k] F_r[k] (k <= n/2, zero above;
// row r of F at r fstride).  tmp holds batch n complex values.
bool fft4_supported(int64_t n);
int fft4_lo_bits(int64_t n);
void fft4_forward_real(const rf_ctx* c, const float* x, float2* out, float2* tmp, cudaStream_t s);
void fft4_inverse(const rf_ctx* c, const float2* in, float2* out, float2* tmp, int batch, cudaStream_t s);
void fft4_inverse_product(const rf_ctx* c, const float2* X, const float2* F, int64_t fstride, float2* out,
                          float2* tmp, int batch, cudaStream_t s);
void real_to_complex_f64(const double* x, double2* out, int64_t n, cudaStream_t s);
void real_to_complex_f32(const float* x, float2* out, int64_t n, cudaStream_t s);
// Host-side FP64 twiddle table exp(-2 pi i m / n), m < n (octant symmetric, accurate).
std::vector<double2> host_twiddles(int64_t n);
// Stage twiddle tables of the block FFTs for B = 2^9 .. 2^14 (float2, concatenated), with
// the entry offset of each block size in off[log2 B].
std::vector<float2> block_fft_tables(int64_t off[16]);

// ---------------------------------------------------------------- MF (mf.cu)
void reference_filters_impl(rf_ctx* c, const double* inv_psd, int32_t nref, const rf_template* refs, void* filt,
                            double* sigma_out, cudaStream_t s);
void mf_filtered_impl(rf_ctx* c, const void* x, int32_t nref, const void* filt, void* z_out, cudaStream_t s);
void mf_reference_impl(rf_ctx* c, const void* x, const double* inv_psd, int32_t nref,
                       const rf_template* refs, void* z_out, double* sigma_out, cudaStream_t s);
void template_fd_impl(rf_ctx* c, const rf_template& t, void* h_out, cudaStream_t s);
// sigma^2 = 4 df sum_band B(f)^2 inv_psd for `count` templates -> out[count] (device, FP64)
void sigma2_impl(rf_ctx* c, const double* inv_psd, int count, double* out, cudaStream_t s);

// ---------------------------------------------------------------- builder (builder.cu)
rf_kernels* build_impl(rf_ctx* c, const rf_template& ref, const rf_template* nbrs, int32_t k,
                       const double* inv_psd, double thr, int relative, int64_t n_build, cudaStream_t s);
rf_kernels* import_impl(rf_ctx* c, int32_t k, const int32_t* lag0, const int32_t* len,
                        const void* taps, bool real);

// ---------------------------------------------------------------- reconstruct
void reconstruct_direct(rf_ctx* c, const void* z_ref, const rf_kernels* kern, void* z_out,
                        int64_t W, float* max_out, int32_t* argmax_out, cudaStream_t s);
void winmax_series(rf_ctx* c, const void* z, int32_t count, int64_t W, float* max_out,
                   int32_t* argmax_out, cudaStream_t s);
// overlap-save (reconstruct_os.cu); FP32 grids, block sizes 512..16384
// Overlap-save layout (block size, partition length) of least modelled cost for kernels of
// the given lengths; block != 0 fixes the block size.
void os_choose_layout(const rf_ctx* c, const std::vector<int>& lengths, int block, bool real, int* B, int* Lp);
// modelled cost (ns, whole GPU) of one layout for kernels of the given lengths
double os_layout_cost(const rf_ctx* c, const std::vector<int>& lengths, int B, int Lp);
// autotune.cu
void autotune_impl(rf_ctx* c, int32_t G, const void* const* z_refs, rf_kernels* const* ks, int64_t W,
                   int32_t flags, int32_t max_os, rf_tune_entry* out, int32_t max_out, int32_t* n_out,
                   cudaStream_t s);
// B = 0 and/or Lp = 0 take the modelled choice.
void os_prepare(rf_ctx* c, rf_kernels* kern, int B, int Lp, cudaStream_t s);
// Several layout buckets: bucket b takes the kernels with cuts[b] <= L < cuts[b + 1]
// (cuts[0] = 0, increasing) and runs with (Bs[b], Lps[b]).
void os_prepare_buckets(rf_ctx* c, rf_kernels* kern, int nb, const int32_t* cuts, const int32_t* Bs,
                        const int32_t* Lps, cudaStream_t s);
// One bucket of a mixed preparation: kernels with cut <= L < next cut run overlap-save (algo
// RF_ALGO_OS; block, part), the tensor-core form (RF_ALGO_GEMM; prec, tile layout block =
// neighbours per group and part = stacked tiles, 0 and 0 for the rule) or the direct sum.
struct BucketSpec {
  int32_t cut, algo, prec, block, part;
};
void os_prepare_forms(rf_ctx* c, rf_kernels* kern, int nb, const BucketSpec* spec, cudaStream_t s);
// two-phase overlap-save (reconstruct_bins.cu): layouts it takes, its plan over a list of items,
// and the launches of a plan (zs_one: the segment spectra of every item, or null for the items'
// own; keys null for the series form into z_out rows)
bool bins_layout_ok(int B, int Lp);
BinsPlan bins_plan(std::vector<OsItem> items, int B, int Lp, bool herm, int64_t n);
// scratch, side stream and events the two-phase launches of block size B need (created outside
// any stream capture)
void bins_prepare_scratch(rf_ctx* c, int B);
void bins_run(rf_ctx* c, const BinsPlan& pl, const OsItem* items_dev, const float2* zs_one, float2* Y,
              float2* z_out, unsigned long long* keys, int64_t W, cudaStream_t s);
size_t os_workspace_bytes(const rf_ctx* c, int32_t k, int64_t W, int Q);
// launches the bounded-wait health check (reconstruct_gemm.cu)
void wait_selftest(rf_ctx* c, cudaStream_t s);
// bytes of the core-matrix records of z_ref used by the tensor-core path at prec (taps padded to LP)
size_t gemm_zplanes_bytes(int64_t n, int64_t LP, int prec);
void reconstruct_os(rf_ctx* c, const void* z_ref, rf_kernels* kern, void* z_out, int64_t W, float* max_out,
                    int32_t* argmax_out, cudaStream_t s);
void reconstruct_batched(rf_ctx* c, int32_t G, const void* const* z_refs, rf_kernels* const* ks, int64_t W,
                         float* max_out, int32_t* argmax_out, cudaStream_t s);
// tensor-core direct form (reconstruct_gemm.cu); kernels of at most gemm_max_len() taps
int gemm_max_len();
// tile layouts: (16, gemm_stacked_shifts(prec)) or (gemm_wide_nj(prec), 1); (0, 0) = the rule
bool gemm_layout_ok(int prec, int nj, int s);
int gemm_stacked_shifts(int prec);
int gemm_wide_nj(int prec);
void gemm_prepare(rf_ctx* c, rf_kernels* kern, int prec, cudaStream_t s);
void reconstruct_gemm(rf_ctx* c, const void* z_ref, rf_kernels* kern, int prec, void* z_out, int64_t W,
                      float* max_out, int32_t* argmax_out, cudaStream_t s);

}  // namespace rf
