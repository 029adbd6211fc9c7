// Streaming over data longer than one segment.  Segments of the context's n samples start at
// s_q = q hop - guard (hop = n - 2 guard, q = 0, 1, ...; data outside [0, total) is zero), so
// their interiors [s_q + guard, s_q + n - guard) tile the stream.  Per segment: the stored-filter
// matched filter of every reference (Sec. II.A), the references' window peaks, and the batched
// reconstruction of their neighbours with fused window peaks (Eqs. 7-8); a window of W samples
// is taken from the segment whose interior holds it, its argmax shifted to a stream index.  The
// circular wrap of a segment reaches only its first and last `guard` samples when guard covers
// the longest template plus the kernels' lag extents.
#include <algorithm>
#include <cstring>
#include <vector>

#include "rf_internal.h"

namespace rf {

namespace {

struct Stream {
  cudaStream_t s = nullptr;
  Stream() { RF_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)); }
  ~Stream() {
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  }
  Stream(const Stream&) = delete;
  Stream& operator=(const Stream&) = delete;
};

struct Event {
  cudaEvent_t e = nullptr;
  Event() { RF_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming)); }
  ~Event() {
    if (e) cudaEventDestroy(e);
  }
  Event(const Event&) = delete;
  Event& operator=(const Event&) = delete;
};

void check_status(rf_status st) {
  if (st != RF_OK) throw Fail{st};  // the callee has recorded the message
}

}  // namespace

// Two staging buffers: while the device works on segment q (on `s`), the host stages segment
// q + 1 and a second stream uploads it, and the host scatters the window peaks of segment q - 1.
// Events order the reuse: an upload into a device buffer waits for the work that last read it,
// the work on a segment waits for its upload, the host waits for a segment's peaks before
// reading them.
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
  const int64_t nseg = (nwt * W + hop - 1) / hop;
  DevBuf* xd = c->st_x;
  DevBuf &zd = c->st_z, &pm = c->st_pm, &pa = c->st_pa;
  for (int i = 0; i < 2; ++i) xd[i].ensure((size_t)n * rsz);
  zd.ensure((size_t)G * n * 2 * rsz);
  pm.ensure(sizeof(float) * (size_t)(all * nws));
  pa.ensure(sizeof(int32_t) * (size_t)(all * nws));
  // pinned block: two strain stagings, two peak-value and two peak-index buffers
  auto up256 = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t bx = up256((size_t)n * rsz), bm = up256(sizeof(float) * (size_t)(all * nws)),
               ba = up256(sizeof(int32_t) * (size_t)(all * nws));
  c->st_pin.ensure(2 * (bx + bm + ba));
  char* pin = static_cast<char*>(c->st_pin.p);
  void* xs[2] = {pin, pin + bx};
  void* hm[2] = {pin + 2 * bx, pin + 2 * bx + bm};
  void* ha[2] = {pin + 2 * (bx + bm), pin + 2 * (bx + bm) + ba};
  Stream up;
  Event up_done[2], work_done[2];
  std::vector<const void*> zp(G);
  for (int g = 0; g < G; ++g) zp[g] = static_cast<const char*>(zd.p) + (size_t)g * n * 2 * rsz;
  const char* xh = static_cast<const char*>(x_host);

  auto upload = [&](int64_t q) {  // stage segment q and start its upload
    const int b = (int)(q & 1);
    const int64_t s0 = q * hop - guard;
    const int64_t a = std::max<int64_t>(0, s0), e = std::min<int64_t>(total, s0 + n);
    RF_CUDA(cudaEventSynchronize(up_done[b].e));  // the staging buffer's previous upload has finished
    std::memset(xs[b], 0, (size_t)n * rsz);
    if (e > a) std::memcpy(static_cast<char*>(xs[b]) + (size_t)(a - s0) * rsz, xh + (size_t)a * rsz, (size_t)(e - a) * rsz);
    RF_CUDA(cudaStreamWaitEvent(up.s, work_done[b].e, 0));  // the device buffer's last reader
    RF_CUDA(cudaMemcpyAsync(xd[b].p, xs[b], (size_t)n * rsz, cudaMemcpyHostToDevice, up.s));
    RF_CUDA(cudaEventRecord(up_done[b].e, up.s));
  };
  auto scatter = [&](int64_t q) {  // window peaks of segment q into the stream's outputs
    const int b = (int)(q & 1);
    RF_CUDA(cudaEventSynchronize(work_done[b].e));
    const int64_t s0 = q * hop - guard;
    const float* m = static_cast<const float*>(hm[b]);
    const int32_t* i = static_cast<const int32_t*>(ha[b]);
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
  };

  upload(0);
  for (int64_t q = 0; q < nseg; ++q) {
    const int b = (int)(q & 1);
    RF_CUDA(cudaStreamWaitEvent(s, up_done[b].e, 0));
    check_status(rf_mf_filtered(c, xd[b].p, G, filt, zd.p, s));
    check_status(rf_winmax(c, zd.p, G, W, pm.as<float>(), pa.as<int32_t>(), s));
    if (rows)
      check_status(rf_reconstruct_batched(c, G, zp.data(), ks, RF_ALGO_AUTO, RF_PREC_NATIVE, W,
                                          pm.as<float>() + G * nws, pa.as<int32_t>() + G * nws, s));
    // the pinned peaks buffer b was last read by the scatter of segment q - 2 (done on the host)
    RF_CUDA(cudaMemcpyAsync(hm[b], pm.p, sizeof(float) * (size_t)(all * nws), cudaMemcpyDeviceToHost, s));
    RF_CUDA(cudaMemcpyAsync(ha[b], pa.p, sizeof(int32_t) * (size_t)(all * nws), cudaMemcpyDeviceToHost, s));
    RF_CUDA(cudaEventRecord(work_done[b].e, s));
    if (q + 1 < nseg) upload(q + 1);
    if (q >= 1) scatter(q - 1);
  }
  scatter(nseg - 1);
}

}  // namespace rf
