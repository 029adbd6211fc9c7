// C ABI entry points: argument validation, dispatch and error reporting.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <memory>
#include <new>

#include "rf_internal.h"

namespace rf {

namespace {
thread_local char g_err[1024] = {0};
}

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

void clear_error() { g_err[0] = 0; }

namespace {
std::atomic<unsigned long long> g_launches{0};
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void DevBuf::ensure(size_t b) {
  if (bytes >= b && p) return;
  release();
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, b);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    set_error("cudaMalloc(%zu bytes) failed: %s", b, cudaGetErrorString(e));
    throw Fail{RF_ENOMEM};
  }
  p = q;
  bytes = b;
}

namespace {

bool is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

// Device pointer check: non-null, 16-byte aligned, and known to CUDA as device or
// managed memory (host pointers are rejected rather than faulting in a kernel).
void check_dev(const void* p, const char* name, bool allow_null = false) {
  if (!p) {
    RF_REQUIRE(allow_null, "%s is NULL", name);
    return;
  }
  RF_REQUIRE(((uintptr_t)p & 15u) == 0, "%s is not 16-byte aligned", name);
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    RF_REQUIRE(false, "%s is not a CUDA device pointer", name);
  }
  RF_REQUIRE(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged,
             "%s is not device memory (memory type %d)", name, (int)at.type);
}

void check_host(const void* p, const char* name) { RF_REQUIRE(p != nullptr, "%s is NULL", name); }

void check_template(const rf_template& t, const char* name) {
  RF_REQUIRE(std::isfinite(t.m1) && std::isfinite(t.m2) && t.m1 > 0 && t.m2 > 0 && t.m1 < 1e4 && t.m2 < 1e4,
             "%s: component masses must be finite and positive", name);
  RF_REQUIRE(std::isfinite(t.tc) && std::isfinite(t.phic), "%s: tc and phic must be finite", name);
}

void check_ctx(const rf_ctx* c) {
  RF_REQUIRE(c != nullptr, "context is NULL");
  int dev = -1;
  RF_CUDA(cudaGetDevice(&dev));
  RF_REQUIRE(dev == c->device, "context belongs to device %d but device %d is current", c->device, dev);
}

template <typename F>
rf_status guard(F&& f) {
  clear_error();
  try {
    f();
    return RF_OK;
  } catch (const Fail& e) {
    return e.st;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return RF_ENOMEM;
  } catch (...) {
    set_error("unexpected internal error");
    return RF_EINVAL;
  }
}

}  // namespace
}  // namespace rf

using namespace rf;

extern "C" {

int32_t rf_version(void) { return RF_ABI_VERSION; }

const char* rf_last_error(void) { return g_err; }

uint64_t rf_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

rf_status rf_create(const rf_grid* grid, rf_ctx** out) {
  return guard([&] {
    RF_REQUIRE(grid != nullptr && out != nullptr, "grid and out must be non-NULL");
    *out = nullptr;
    const rf_grid g = *grid;
    RF_REQUIRE(is_pow2(g.n) && g.n >= 256 && g.n <= (int64_t(1) << 24), "n=%lld must be a power of two in [2^8, 2^24]",
               (long long)g.n);
    RF_REQUIRE(std::isfinite(g.fs) && g.fs > 0, "fs must be positive");
    RF_REQUIRE(std::isfinite(g.f_low) && std::isfinite(g.f_high) && g.f_low > 0 && g.f_low < g.f_high,
               "need 0 < f_low < f_high");
    RF_REQUIRE(std::isfinite(g.df_high) && g.df_high >= 0 && std::isfinite(g.df_low_max) && g.df_low_max >= 0,
               "taper widths must be non-negative");
    RF_REQUIRE(g.f_high + g.df_high <= 0.5 * g.fs * (1 + 1e-12), "f_high + df_high must not exceed fs/2");
    RF_REQUIRE(g.pn_order >= 0 && g.pn_order <= 7, "pn_order must be 0..7");
    RF_REQUIRE(g.dtype == RF_F64 || g.dtype == RF_F32, "dtype must be RF_F64 or RF_F32");
    std::unique_ptr<rf_ctx> c(new rf_ctx());
    c->g = g;
    c->n = g.n;
    RF_CUDA(cudaGetDevice(&c->device));
    RF_CUDA(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device));
    const int64_t n = g.n;
    const std::vector<double2> tw = host_twiddles(n);
    c->tw64.ensure(sizeof(double2) * n);
    RF_CUDA(cudaMemcpy(c->tw64.p, tw.data(), sizeof(double2) * n, cudaMemcpyHostToDevice));
    std::vector<float2> tw32((size_t)n);
    for (int64_t m = 0; m < n; ++m) tw32[m] = make_float2((float)tw[m].x, (float)tw[m].y);
    c->tw32.ensure(sizeof(float2) * n);
    RF_CUDA(cudaMemcpy(c->tw32.p, tw32.data(), sizeof(float2) * n, cudaMemcpyHostToDevice));
    if (g.dtype == RF_F32 && fft4_supported(n)) {
      // four-step FFT twiddles: the low table, then every 2^lo-th entry
      const int lo = fft4_lo_bits(n);
      std::vector<float2> t4((size_t)((int64_t(1) << lo) + (n >> lo)));
      for (int64_t m = 0; m < (int64_t(1) << lo); ++m) t4[m] = tw32[m];
      for (int64_t m = 0; m < (n >> lo); ++m) t4[(int64_t(1) << lo) + m] = tw32[m << lo];
      c->tw4.ensure(sizeof(float2) * t4.size());
      RF_CUDA(cudaMemcpy(c->tw4.p, t4.data(), sizeof(float2) * t4.size(), cudaMemcpyHostToDevice));
      c->tw4_lo_bits = lo;
    }
    // stage twiddle tables of the overlap-save block FFTs
    const std::vector<float2> twb = block_fft_tables(c->twb_off);
    c->twb32.ensure(sizeof(float2) * twb.size());
    RF_CUDA(cudaMemcpy(c->twb32.p, twb.data(), sizeof(float2) * twb.size(), cudaMemcpyHostToDevice));
    const size_t esz = g.dtype == RF_F64 ? sizeof(double2) : sizeof(float2);
    c->xf.ensure(esz * n);
    c->fa.ensure(esz * n);
    c->fb.ensure(esz * n);
    c->red.ensure(sizeof(double) * 1024);
    c->status.ensure(sizeof(int) * 4);
    RF_CUDA(cudaMemset(c->status.p, 0, sizeof(int) * 4));
    *out = c.release();
  });
}

void rf_destroy(rf_ctx* ctx) {
  if (!ctx) return;
  cudaDeviceSynchronize();
  delete ctx;
}

rf_status rf_reserve(rf_ctx* ctx, int32_t k_max, int64_t* bytes_out) {
  return guard([&] {
    check_ctx(ctx);
    RF_REQUIRE(k_max >= 0, "k_max must be non-negative");
    // overlap-save segment spectra plus packed window keys for windows of >= 16 samples
    const size_t bytes = os_workspace_bytes(ctx, k_max, 16, 8);  // the largest partition ratio
    ctx->scratch.ensure(bytes);
    // core-matrix records of z_ref for the tensor-core path, for taps up to the segment length
    const int64_t lp_max = std::min<int64_t>(ctx->n, gemm_max_len()) + 128;
    const size_t planes = std::max(gemm_zplanes_bytes(ctx->n, lp_max, RF_PREC_BF16X9),
                                   gemm_zplanes_bytes(ctx->n, lp_max, RF_PREC_3XTF32));
    ctx->scratch2.ensure(planes);
    ctx->reserved = bytes;
    if (bytes_out) *bytes_out = (int64_t)(bytes + planes);
  });
}

rf_status rf_template_fd(rf_ctx* ctx, const rf_template* tmpl, void* h_out, rf_stream stream) {
  return guard([&] {
    check_ctx(ctx);
    check_host(tmpl, "tmpl");
    check_template(*tmpl, "tmpl");
    check_dev(h_out, "h_out");
    template_fd_impl(ctx, *tmpl, h_out, (cudaStream_t)stream);
  });
}

rf_status rf_mf_reference(rf_ctx* ctx, const void* x, const double* inv_psd, int32_t nref, const rf_template* refs,
                          void* z_out, double* sigma_out, rf_stream stream) {
  return guard([&] {
    check_ctx(ctx);
    RF_REQUIRE(nref >= 1, "nref must be >= 1");
    check_host(refs, "refs");
    for (int r = 0; r < nref; ++r) check_template(refs[r], "refs[r]");
    check_dev(x, "x");
    check_dev(inv_psd, "inv_psd");
    check_dev(z_out, "z_out");
    check_dev(sigma_out, "sigma_out", true);
    mf_reference_impl(ctx, x, inv_psd, nref, refs, z_out, sigma_out, (cudaStream_t)stream);
  });
}

rf_status rf_reference_filters(rf_ctx* ctx, const double* inv_psd, int32_t nref, const rf_template* refs,
                               void* filt_out, double* sigma_out, rf_stream stream) {
  return guard([&] {
    check_ctx(ctx);
    RF_REQUIRE(nref >= 1, "nref must be >= 1");
    check_host(refs, "refs");
    for (int r = 0; r < nref; ++r) check_template(refs[r], "refs[r]");
    check_dev(inv_psd, "inv_psd");
    check_dev(filt_out, "filt_out");
    check_dev(sigma_out, "sigma_out", true);
    reference_filters_impl(ctx, inv_psd, nref, refs, filt_out, sigma_out, (cudaStream_t)stream);
  });
}

rf_status rf_mf_filtered(rf_ctx* ctx, const void* x, int32_t nref, const void* filt, void* z_out, rf_stream stream) {
  return guard([&] {
    check_ctx(ctx);
    RF_REQUIRE(nref >= 1, "nref must be >= 1");
    RF_REQUIRE(ctx->n >= 16, "the stored-filter form needs n >= 16");
    check_dev(x, "x");
    check_dev(filt, "filt");
    check_dev(z_out, "z_out");
    mf_filtered_impl(ctx, x, nref, filt, z_out, (cudaStream_t)stream);
  });
}

rf_status rf_build_ratio_kernels(rf_ctx* ctx, const rf_template* ref, const rf_template* nbrs, int32_t k,
                                 const double* inv_psd, double threshold, int32_t relative, int64_t n_build,
                                 rf_kernels** out, rf_stream stream) {
  return guard([&] {
    RF_REQUIRE(out != nullptr, "out is NULL");
    *out = nullptr;
    check_ctx(ctx);
    check_host(ref, "ref");
    check_template(*ref, "ref");
    RF_REQUIRE(k >= 0, "k must be >= 0");
    if (k) check_host(nbrs, "nbrs");
    for (int j = 0; j < k; ++j) check_template(nbrs[j], "nbrs[j]");
    check_dev(inv_psd, "inv_psd");
    RF_REQUIRE(std::isfinite(threshold) && threshold >= 0, "threshold must be finite and >= 0");
    RF_REQUIRE(relative >= 0 && relative <= (RF_TRUNC_RELATIVE | RF_TRUNC_ANALYTIC | RF_KERNEL_REAL),
               "relative=%d: flags are RF_TRUNC_RELATIVE | RF_TRUNC_ANALYTIC | RF_KERNEL_REAL", relative);
    RF_REQUIRE(!(relative & RF_TRUNC_ANALYTIC) || threshold > 0, "analytic truncation needs threshold > 0");
    RF_REQUIRE(n_build == 0 || n_build == -1 ||
                   (n_build >= 16 && n_build <= ctx->n && (n_build & (n_build - 1)) == 0),
               "n_build=%lld must be 0, -1 or a power of two in [16, n]", (long long)n_build);
    *out = build_impl(ctx, *ref, nbrs, k, inv_psd, threshold, relative, n_build, (cudaStream_t)stream);
  });
}

static void import_checked(rf_ctx* ctx, int32_t k, const int32_t* lag0, const int32_t* len, const void* taps,
                           bool real, rf_kernels** out) {
  {  // argument checks, then the copy (thrown failures become the caller's status)
    RF_REQUIRE(out != nullptr, "out is NULL");
    *out = nullptr;
    check_ctx(ctx);
    RF_REQUIRE(k >= 0, "k must be >= 0");
    int64_t total = 0;
    if (k) {
      check_host(lag0, "lag0");
      check_host(len, "len");
      for (int j = 0; j < k; ++j) {
        RF_REQUIRE(len[j] >= 0 && len[j] <= ctx->n, "len[%d]=%d outside [0, n]", j, len[j]);
        RF_REQUIRE(lag0[j] > -ctx->n && lag0[j] < ctx->n, "lag0[%d]=%d outside (-n, n)", j, lag0[j]);
        total += len[j];
      }
    }
    if (total) check_host(taps, "taps");
    *out = import_impl(ctx, k, lag0, len, taps, real);
  }
}

rf_status rf_kernels_import(rf_ctx* ctx, int32_t k, const int32_t* lag0, const int32_t* len, const void* taps,
                            rf_kernels** out) {
  return guard([&] { import_checked(ctx, k, lag0, len, taps, false, out); });
}

rf_status rf_kernels_import_real(rf_ctx* ctx, int32_t k, const int32_t* lag0, const int32_t* len, const void* taps,
                                 rf_kernels** out) {
  return guard([&] { import_checked(ctx, k, lag0, len, taps, true, out); });
}

rf_status rf_kernels_is_real(const rf_kernels* kern, int32_t* real) {
  return guard([&] {
    RF_REQUIRE(kern != nullptr && real != nullptr, "kern and real must be non-NULL");
    *real = kern->real ? 1 : 0;
  });
}

rf_status rf_kernels_info(const rf_kernels* kern, int32_t* k, const int32_t** len, const int32_t** lag0,
                          const int64_t** offset, const double** df_low, const void** taps_dev) {
  return guard([&] {
    RF_REQUIRE(kern != nullptr, "kern is NULL");
    if (k) *k = kern->k;
    if (len) *len = kern->len.data();
    if (lag0) *lag0 = kern->lag0.data();
    if (offset) *offset = kern->offset.data();
    if (df_low) *df_low = kern->df_low.data();
    if (taps_dev) *taps_dev = kern->taps.p;
  });
}

rf_status rf_kernels_prepare(rf_ctx* ctx, rf_kernels* kern, int32_t block, int32_t part, rf_stream stream) {
  return guard([&] {
    check_ctx(ctx);
    RF_REQUIRE(kern != nullptr, "kern is NULL");
    RF_REQUIRE(kern->n == ctx->n && kern->dtype == ctx->g.dtype, "kernels were made for another grid");
    if (ctx->g.dtype != RF_F32 || ctx->n < 512) {
      set_error("overlap-save needs an RF_F32 grid with n >= 512");
      throw Fail{RF_EUNSUPPORTED};
    }
    RF_REQUIRE(block >= 0 && part >= 0, "block and part must be non-negative");
    os_prepare(ctx, kern, block, part, (cudaStream_t)stream);
  });
}

rf_status rf_kernels_prepare_buckets(rf_ctx* ctx, rf_kernels* kern, int32_t nb, const int32_t* cuts,
                                     const int32_t* blocks, const int32_t* parts, rf_stream stream) {
  return guard([&] {
    check_ctx(ctx);
    RF_REQUIRE(kern != nullptr, "kern is NULL");
    RF_REQUIRE(kern->n == ctx->n && kern->dtype == ctx->g.dtype, "kernels were made for another grid");
    if (ctx->g.dtype != RF_F32 || ctx->n < 512) {
      set_error("overlap-save needs an RF_F32 grid with n >= 512");
      throw Fail{RF_EUNSUPPORTED};
    }
    RF_REQUIRE(nb >= 1 && nb <= 8, "nb must be in [1, 8]");
    check_host(cuts, "cuts");
    check_host(blocks, "blocks");
    check_host(parts, "parts");
    os_prepare_buckets(ctx, kern, nb, cuts, blocks, parts, (cudaStream_t)stream);
  });
}

rf_status rf_kernels_prepare_forms(rf_ctx* ctx, rf_kernels* kern, int32_t nb, const int32_t* cuts,
                                   const int32_t* algos, const int32_t* precs, const int32_t* blocks,
                                   const int32_t* parts, rf_stream stream) {
  return guard([&] {
    check_ctx(ctx);
    RF_REQUIRE(kern != nullptr, "kern is NULL");
    RF_REQUIRE(kern->n == ctx->n && kern->dtype == ctx->g.dtype, "kernels were made for another grid");
    if (ctx->g.dtype != RF_F32 || ctx->n < 512) {
      set_error("bucketed preparation needs an RF_F32 grid with n >= 512");
      throw Fail{RF_EUNSUPPORTED};
    }
    RF_REQUIRE(nb >= 1 && nb <= 8, "nb must be in [1, 8]");
    check_host(cuts, "cuts");
    check_host(algos, "algos");
    check_host(precs, "precs");
    check_host(blocks, "blocks");
    check_host(parts, "parts");
    std::vector<BucketSpec> spec(nb);
    for (int b = 0; b < nb; ++b) spec[b] = BucketSpec{cuts[b], algos[b], precs[b], blocks[b], parts[b]};
    os_prepare_forms(ctx, kern, nb, spec.data(), (cudaStream_t)stream);
  });
}

rf_status rf_kernels_bucket_forms(const rf_kernels* kern, int32_t max_nb, int32_t* algos, int32_t* precs,
                                  int32_t* nb) {
  return guard([&] {
    RF_REQUIRE(kern != nullptr, "kern is NULL");
    RF_REQUIRE(max_nb >= 0, "max_nb must be >= 0");
    const int cnt = kern->os_ready ? (int)kern->os_buckets.size() : 0;
    for (int b = 0; b < std::min(cnt, (int)max_nb); ++b) {
      if (algos) algos[b] = kern->os_buckets[b].algo;
      if (precs) precs[b] = kern->os_buckets[b].prec;
    }
    if (nb) *nb = std::min(cnt, (int)max_nb);
  });
}

rf_status rf_kernels_os_buckets(const rf_kernels* kern, int32_t max_nb, int32_t* cuts, int32_t* blocks,
                                int32_t* parts, int32_t* nb) {
  return guard([&] {
    RF_REQUIRE(kern != nullptr, "kern is NULL");
    RF_REQUIRE(max_nb >= 0, "max_nb must be >= 0");
    const int cnt = kern->os_ready ? (int)kern->os_buckets.size() : 0;
    for (int b = 0; b < std::min(cnt, (int)max_nb); ++b) {
      const OsBucket& o = kern->os_buckets[b];
      const bool os_like = o.algo == RF_ALGO_OS || o.algo == RF_ALGO_OS_BINS;
      if (cuts) cuts[b] = o.cut_lo;
      if (blocks) blocks[b] = os_like ? o.B : o.gemm_nj;
      if (parts) parts[b] = os_like ? o.Lp : o.gemm_s;
    }
    if (nb) *nb = std::min(cnt, (int)max_nb);
  });
}

rf_status rf_kernels_grids(const rf_kernels* kern, const int64_t** grids) {
  return guard([&] {
    RF_REQUIRE(kern != nullptr, "kern is NULL");
    RF_REQUIRE(grids != nullptr, "grids is NULL");
    *grids = kern->grid.data();
  });
}

rf_status rf_kernels_os_layout(const rf_kernels* kern, int32_t* block, int32_t* part) {
  return guard([&] {
    RF_REQUIRE(kern != nullptr, "kern is NULL");
    if (block) *block = kern->os_ready ? kern->os_B : 0;
    if (part) *part = kern->os_ready ? kern->os_Lp : 0;
  });
}

rf_status rf_stream_winmax(rf_ctx* ctx, const void* x_host, int64_t total, int32_t G, const void* filt,
                           rf_kernels* const* ks, int64_t W, int64_t guard_samples, float* ref_max, int64_t* ref_arg,
                           float* nbr_max, int64_t* nbr_arg, rf_stream stream) {
  return guard([&] {
    check_ctx(ctx);
    RF_REQUIRE(G >= 1 && ks != nullptr, "G must be >= 1 and ks non-NULL");
    RF_REQUIRE(W >= 1 && ctx->n % W == 0, "W=%lld must divide n", (long long)W);
    RF_REQUIRE(guard_samples >= 0 && guard_samples % W == 0 && 2 * guard_samples < ctx->n,
               "guard_samples=%lld: a multiple of W below n/2", (long long)guard_samples);
    RF_REQUIRE(total >= W, "total=%lld: at least one window", (long long)total);
    check_host(x_host, "x_host");
    check_dev(filt, "filt");
    check_host(ref_max, "ref_max");
    check_host(ref_arg, "ref_arg");
    int64_t rows = 0;
    for (int g = 0; g < G; ++g) {
      RF_REQUIRE(ks[g] != nullptr, "ks[%d] is NULL", g);
      rows += ks[g]->k;
    }
    if (rows) {
      check_host(nbr_max, "nbr_max");
      check_host(nbr_arg, "nbr_arg");
    }
    stream_winmax_impl(ctx, x_host, total, G, filt, ks, W, guard_samples, ref_max, ref_arg, nbr_max, nbr_arg,
                       (cudaStream_t)stream);
  });
}

rf_status rf_bank_structure(const rf_template* bank, int32_t count, double f_low, int32_t pn_order,
                            double max_spread, int32_t max_size, int32_t* set_of, int32_t* ref_of_set,
                            int32_t* n_sets, double* duration_out) {
  return guard([&] {
    RF_REQUIRE(n_sets != nullptr, "n_sets is NULL");
    RF_REQUIRE(count >= 0, "count must be >= 0");
    RF_REQUIRE(std::isfinite(f_low) && f_low > 0, "f_low must be positive");
    RF_REQUIRE(pn_order >= 0 && pn_order <= 7, "pn_order must be in 0..7");
    RF_REQUIRE(std::isfinite(max_spread) && max_spread > 0, "max_spread must be positive");
    RF_REQUIRE(max_size >= 1, "max_size must be >= 1");
    if (count > 0) {
      RF_REQUIRE(bank != nullptr && set_of != nullptr && ref_of_set != nullptr, "bank or outputs NULL");
      for (int i = 0; i < count; ++i) check_template(bank[i], "bank[i]");
    }
    bank_structure_impl(bank, count, f_low, pn_order, max_spread, max_size, set_of, ref_of_set, n_sets,
                        duration_out);
  });
}

rf_status rf_kernels_gemm_layout(const rf_kernels* kern, int32_t* out) {
  return guard([&] {
    RF_REQUIRE(kern != nullptr, "kern is NULL");
    RF_REQUIRE(out != nullptr, "out is NULL");
    const bool r = kern->gemm_ready;
    out[0] = r ? kern->gemm_prec : 0;
    out[1] = r ? kern->gemm_NJ : 0;
    out[2] = r ? kern->gemm_S : 0;
    out[3] = r ? kern->gemm_KC : 0;
    out[4] = r ? kern->gemm_NCK : 0;
    out[5] = r ? kern->gemm_LP : 0;
  });
}

rf_status rf_kernels_copy_taps(const rf_kernels* kern, void* dst, rf_stream stream) {
  return guard([&] {
    RF_REQUIRE(kern != nullptr, "kern is NULL");
    const size_t bytes = (size_t)kern->offset[kern->k] * tap_bytes(kern);
    if (!bytes) return;
    check_dev(dst, "dst");
    RF_CUDA(cudaMemcpyAsync(dst, kern->taps.p, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  });
}

void rf_kernels_free(rf_kernels* kern) {
  if (!kern) return;
  cudaDeviceSynchronize();
  delete kern;
}

// Validates a reconstruction call and resolves RF_ALGO_AUTO: the autotuned form of the kernel
// set (with its precision) when there is one, else overlap-save on FP32 grids with n >= 512 and
// the direct sum otherwise.
static int check_recon(rf_ctx* ctx, const void* z_ref, const rf_kernels* kern, int32_t algo, int32_t& prec) {
  check_ctx(ctx);
  RF_REQUIRE(kern != nullptr, "kern is NULL");
  RF_REQUIRE(kern->n == ctx->n && kern->dtype == ctx->g.dtype, "kernels were made for another grid");
  check_dev(z_ref, "z_ref");
  RF_REQUIRE(algo == RF_ALGO_AUTO || algo == RF_ALGO_DIRECT || algo == RF_ALGO_OS || algo == RF_ALGO_GEMM,
             "unknown algo %d", algo);
  RF_REQUIRE(prec >= RF_PREC_NATIVE && prec <= RF_PREC_3XTF32, "unknown prec %d", prec);
  if (algo == RF_ALGO_AUTO && kern->tuned_algo && prec == RF_PREC_NATIVE) {
    algo = kern->tuned_algo;
    prec = kern->tuned_prec;
  }
  if (algo == RF_ALGO_GEMM) {
    RF_REQUIRE(prec != RF_PREC_NATIVE, "the tensor-core form needs a split precision (RF_PREC_BF16* or RF_PREC_3XTF32)");
    if (kern->max_len > gemm_max_len() || ctx->n % 128 != 0) {
      set_error("the tensor-core form takes kernels of at most %d taps and n a multiple of 128", gemm_max_len());
      throw Fail{RF_EUNSUPPORTED};
    }
    return algo;
  }
  RF_REQUIRE(prec == RF_PREC_NATIVE, "split precisions apply to RF_ALGO_GEMM only");
  const bool os_ok = ctx->g.dtype == RF_F32 && ctx->n >= 512;
  if (algo == RF_ALGO_OS && !os_ok) {
    set_error("overlap-save needs an RF_F32 grid with n >= 512");
    throw Fail{RF_EUNSUPPORTED};
  }
  if (algo == RF_ALGO_AUTO) algo = os_ok ? RF_ALGO_OS : RF_ALGO_DIRECT;
  return algo;
}

rf_status rf_reconstruct(rf_ctx* ctx, const void* z_ref, const rf_kernels* kern, int32_t algo, int32_t prec,
                         void* z_out, rf_stream stream) {
  return guard([&] {
    const int a = check_recon(ctx, z_ref, kern, algo, prec);
    if (kern->k) check_dev(z_out, "z_out");
    if (a == RF_ALGO_OS)
      reconstruct_os(ctx, z_ref, const_cast<rf_kernels*>(kern), z_out, 0, nullptr, nullptr, (cudaStream_t)stream);
    else if (a == RF_ALGO_GEMM)
      reconstruct_gemm(ctx, z_ref, const_cast<rf_kernels*>(kern), prec, z_out, 0, nullptr, nullptr,
                       (cudaStream_t)stream);
    else
      reconstruct_direct(ctx, z_ref, kern, z_out, 0, nullptr, nullptr, (cudaStream_t)stream);
  });
}

rf_status rf_reconstruct_winmax(rf_ctx* ctx, const void* z_ref, const rf_kernels* kern, int32_t algo, int32_t prec,
                                int64_t W, float* max_out, int32_t* argmax_out, rf_stream stream) {
  return guard([&] {
    const int a = check_recon(ctx, z_ref, kern, algo, prec);
    RF_REQUIRE(W >= 1 && W <= ctx->n, "W=%lld must be in [1, n]", (long long)W);
    if (kern->k) {
      check_dev(max_out, "max_out");
      check_dev(argmax_out, "argmax_out");
    }
    if (a == RF_ALGO_OS)
      reconstruct_os(ctx, z_ref, const_cast<rf_kernels*>(kern), nullptr, W, max_out, argmax_out,
                     (cudaStream_t)stream);
    else if (a == RF_ALGO_GEMM)
      reconstruct_gemm(ctx, z_ref, const_cast<rf_kernels*>(kern), prec, nullptr, W, max_out, argmax_out,
                       (cudaStream_t)stream);
    else
      reconstruct_direct(ctx, z_ref, kern, nullptr, W, max_out, argmax_out, (cudaStream_t)stream);
  });
}

rf_status rf_reconstruct_batched(rf_ctx* ctx, int32_t G, const void* const* z_refs, rf_kernels* const* ks,
                                 int32_t algo, int32_t prec, int64_t W, float* max_out, int32_t* argmax_out,
                                 rf_stream stream) {
  return guard([&] {
    check_ctx(ctx);
    RF_REQUIRE(G >= 1, "G must be >= 1");
    RF_REQUIRE(z_refs != nullptr && ks != nullptr, "z_refs and ks must be non-NULL host arrays");
    RF_REQUIRE(W >= 1 && W <= ctx->n, "W=%lld must be in [1, n]", (long long)W);
    int64_t rows = 0;
    int a = RF_ALGO_AUTO;
    int32_t pa = prec;
    for (int g = 0; g < G; ++g) {
      RF_REQUIRE(ks[g] != nullptr, "ks[%d] is NULL", g);
      int32_t pg = prec;
      const int ag = check_recon(ctx, z_refs[g], ks[g], algo, pg);
      RF_REQUIRE(g == 0 || (ag == a && pg == pa),
                 "the groups resolve to different forms (tune them together with rf_autotune)");
      a = ag;
      pa = pg;
      rows += ks[g]->k;
    }
    prec = pa;
    if (!rows) return;
    check_dev(max_out, "max_out");
    check_dev(argmax_out, "argmax_out");
    if (a == RF_ALGO_OS) {
      reconstruct_batched(ctx, G, z_refs, ks, W, max_out, argmax_out, (cudaStream_t)stream);
      return;
    }
    const int64_t nw = (ctx->n + W - 1) / W;
    int64_t row = 0;
    for (int g = 0; g < G; ++g) {
      if (ks[g]->k) {
        if (a == RF_ALGO_GEMM)
          reconstruct_gemm(ctx, z_refs[g], ks[g], prec, nullptr, W, max_out + row * nw, argmax_out + row * nw,
                           (cudaStream_t)stream);
        else
          reconstruct_direct(ctx, z_refs[g], ks[g], nullptr, W, max_out + row * nw, argmax_out + row * nw,
                             (cudaStream_t)stream);
      }
      row += ks[g]->k;
    }
  });
}

rf_status rf_autotune(rf_ctx* ctx, int32_t G, const void* const* z_refs, rf_kernels* const* ks, int64_t W,
                      int32_t flags, int32_t max_os, rf_tune_entry* out, int32_t max_out, int32_t* n_out,
                      rf_stream stream) {
  return guard([&] {
    check_ctx(ctx);
    RF_REQUIRE(G >= 1, "G must be >= 1");
    RF_REQUIRE(z_refs != nullptr && ks != nullptr, "z_refs and ks must be non-NULL host arrays");
    RF_REQUIRE(W >= 1 && W <= ctx->n, "W=%lld must be in [1, n]", (long long)W);
    RF_REQUIRE(max_out >= 0 && max_os >= 0, "max_out and max_os must be >= 0");
    RF_REQUIRE((flags & ~RF_TUNE_ALLOW_SPLIT) == 0, "unknown flags %d", flags);
    for (int g = 0; g < G; ++g) {
      RF_REQUIRE(ks[g] != nullptr, "ks[%d] is NULL", g);
      RF_REQUIRE(ks[g]->real == ks[0]->real, "the kernel sets of a batch are all complex or all real-form");
      RF_REQUIRE(ks[g]->n == ctx->n && ks[g]->dtype == ctx->g.dtype, "kernels were made for another grid");
      check_dev(z_refs[g], "z_refs[g]");
    }
    autotune_impl(ctx, G, z_refs, ks, W, flags, max_os, out, max_out, n_out, (cudaStream_t)stream);
  });
}

rf_status rf_selftest_bounded_wait(rf_ctx* ctx, rf_stream stream) {
  return guard([&] {
    check_ctx(ctx);
    wait_selftest(ctx, (cudaStream_t)stream);
  });
}

rf_status rf_device_status(rf_ctx* ctx) {
  rf_status out = RF_OK;
  const rf_status st = guard([&] {
    check_ctx(ctx);
    RF_CUDA(cudaDeviceSynchronize());
    int v = 0;
    RF_CUDA(cudaMemcpy(&v, ctx->status.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (v) {
      RF_CUDA(cudaMemset(ctx->status.p, 0, sizeof(int)));
      set_error("a bounded device-side wait ran out (status %d)", v);
      out = (rf_status)v;
    }
  });
  return st != RF_OK ? st : out;
}

rf_status rf_winmax(rf_ctx* ctx, const void* z, int32_t count, int64_t W, float* max_out, int32_t* argmax_out,
                    rf_stream stream) {
  return guard([&] {
    check_ctx(ctx);
    RF_REQUIRE(count >= 0, "count must be >= 0");
    RF_REQUIRE(W >= 1 && W <= ctx->n, "W=%lld must be in [1, n]", (long long)W);
    if (!count) return;
    check_dev(z, "z");
    check_dev(max_out, "max_out");
    check_dev(argmax_out, "argmax_out");
    winmax_series(ctx, z, count, W, max_out, argmax_out, (cudaStream_t)stream);
  });
}

}  // extern "C"
