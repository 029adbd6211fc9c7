// Streaming over data longer than one segment.  Segments of the context's n samples start at
// s_q = q hop - guard (hop = n - 2 guard, q = 0, 1, ...; data outside [0, total) is zero), so
// their interiors [s_q + guard, s_q + n - guard) tile the stream.  Per segment: the stored-filter
// matched filter of every reference (Sec. II.A), the references' window peaks, and the batched
// reconstruction of their neighbours with fused window peaks (Eqs. 7-8); a window of W samples
// is taken from the segment whose interior holds it, its argmax shifted to a stream index.  The
// circular wrap of a segment reaches only its first and last `guard` samples when guard covers
// the longest template plus the kernels' lag extents.
#include <cstring>
#include <vector>

#include "rf_internal.h"

namespace rf {

namespace {

struct PinnedBuf {
  void* p = nullptr;
  explicit PinnedBuf(size_t b) { RF_CUDA(cudaMallocHost(&p, b)); }
  ~PinnedBuf() {
    if (p) cudaFreeHost(p);
  }
  PinnedBuf(const PinnedBuf&) = delete;
  PinnedBuf& operator=(const PinnedBuf&) = delete;
};

void check_status(rf_status st) {
  if (st != RF_OK) throw Fail{st};  // the callee has recorded the message
}

}  // namespace

void stream_winmax_impl(rf_ctx* c, const void* x_host, int64_t total, int32_t G, const void* filt,
                        rf_kernels* const* ks, int64_t W, int64_t guard, float* ref_max, int64_t* ref_arg,
                        float* nbr_max, int64_t* nbr_arg, cudaStream_t s) {
  const int64_t n = c->n;
  const size_t rsz = c->g.dtype == RF_F64 ? sizeof(double) : sizeof(float);
  const int64_t hop = n - 2 * guard;
  const int64_t nws = n / W, nwt = total / W;
  int64_t rows = 0;
  for (int g = 0; g < G; ++g) rows += ks[g]->k;
  const int64_t all = G + rows;
  DevBuf xd, zd, pm, pa;
  xd.ensure((size_t)n * rsz);
  zd.ensure((size_t)G * n * 2 * rsz);
  pm.ensure(sizeof(float) * (size_t)(all * nws));
  pa.ensure(sizeof(int32_t) * (size_t)(all * nws));
  PinnedBuf xs((size_t)n * rsz), hm(sizeof(float) * (size_t)(all * nws)), ha(sizeof(int32_t) * (size_t)(all * nws));
  std::vector<const void*> zp(G);
  for (int g = 0; g < G; ++g) zp[g] = static_cast<const char*>(zd.p) + (size_t)g * n * 2 * rsz;
  const char* xh = static_cast<const char*>(x_host);
  for (int64_t q = 0; q * hop < nwt * W; ++q) {
    const int64_t s0 = q * hop - guard;
    // the segment's samples, zero outside the stream
    const int64_t a = std::max<int64_t>(0, s0), b = std::min<int64_t>(total, s0 + n);
    std::memset(xs.p, 0, (size_t)n * rsz);
    if (b > a) std::memcpy(static_cast<char*>(xs.p) + (size_t)(a - s0) * rsz, xh + (size_t)a * rsz, (size_t)(b - a) * rsz);
    RF_CUDA(cudaMemcpyAsync(xd.p, xs.p, (size_t)n * rsz, cudaMemcpyHostToDevice, s));
    check_status(rf_mf_filtered(c, xd.p, G, filt, zd.p, s));
    check_status(rf_winmax(c, zd.p, G, W, pm.as<float>(), pa.as<int32_t>(), s));
    if (rows)
      check_status(rf_reconstruct_batched(c, G, zp.data(), ks, RF_ALGO_AUTO, RF_PREC_NATIVE, W,
                                          pm.as<float>() + G * nws, pa.as<int32_t>() + G * nws, s));
    RF_CUDA(cudaMemcpyAsync(hm.p, pm.p, sizeof(float) * (size_t)(all * nws), cudaMemcpyDeviceToHost, s));
    RF_CUDA(cudaMemcpyAsync(ha.p, pa.p, sizeof(int32_t) * (size_t)(all * nws), cudaMemcpyDeviceToHost, s));
    RF_CUDA(cudaStreamSynchronize(s));  // the staging buffers are rewritten by the next segment
    const float* m = static_cast<const float*>(hm.p);
    const int32_t* i = static_cast<const int32_t*>(ha.p);
    for (int64_t wl = guard / W; wl < (n - guard) / W; ++wl) {
      const int64_t w = (s0 + wl * W) / W;  // s0 + guard is a multiple of W
      if (w < 0 || w >= nwt) continue;
      for (int64_t r = 0; r < all; ++r) {
        const float v = m[r * nws + wl];
        const int64_t at = s0 + i[r * nws + wl];
        if (r < G) {
          ref_max[r * nwt + w] = v;
          ref_arg[r * nwt + w] = at;
        } else {
          nbr_max[(r - G) * nwt + w] = v;
          nbr_arg[(r - G) * nwt + w] = at;
        }
      }
    }
  }
}

}  // namespace rf
