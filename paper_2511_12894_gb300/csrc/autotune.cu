// Autotuner: picks, for a batch of kernel sets, the reconstruction form and its shape by timing
// candidates on the device.  Candidates: overlap-save layouts (block size B, partition length
// Lp; the cost model of reconstruct_os.cu ranks them and the best few are timed), two-bucket
// overlap-save (short kernels with their own layout, the rest with the fastest single one), the
// tensor-core form at the cheapest split precision that meets the FP32-equivalent accuracy
// (bf16x6) in both of its tile layouts when the kernels are short enough for it to compete,
// mixed forms (the tensor-core form for the shortest kernels, the fastest overlap-save layout for
// the rest, within one call), and the direct sum for short kernels.  Each candidate runs the fused window-peak
// form once to warm up and then three times between CUDA events; the fastest wins and is
// recorded in every kernel set, so that RF_ALGO_AUTO follows it.
#include <algorithm>
#include <vector>

#include "rf_internal.h"

namespace rf {

namespace {

struct Cand {
  int algo, block, part, prec;
  double model;
  int cut = 0, block2 = 0, part2 = 0;  // two buckets: (algo, block, part) below cut, (algo2, block2, part2) above
  int algo2 = RF_ALGO_OS;
  int cut3 = 0, block3 = 0, part3 = 0, algo3 = RF_ALGO_OS;  // a third bucket from cut3 on
};

// layouts of least modelled cost for kernels of the given lengths
std::vector<Cand> os_candidates_for(const rf_ctx* c, const std::vector<int>& all, int max_os, bool real) {
  std::vector<Cand> out;
  for (int B = 512; B <= 32768; B *= 2) {  // 32768: the CTA-pair layout (partitions B/2 or B/4)
    if (B > c->n || (real && B == 32768)) continue;  // real-form sets: single-CTA blocks only
    for (int Q = 2; Q <= (B == 32768 ? 4 : 8); Q *= 2)
      out.push_back(Cand{RF_ALGO_OS, B, B / Q, RF_PREC_NATIVE, os_layout_cost(c, all, B, B / Q)});
  }
  std::sort(out.begin(), out.end(), [](const Cand& a, const Cand& b) { return a.model < b.model; });
  if ((int)out.size() > max_os) out.resize(max_os);
  return out;
}

// the same over all kernel lengths of the batch
std::vector<Cand> os_candidates(const rf_ctx* c, int G, rf_kernels* const* ks, int max_os) {
  std::vector<int> all;
  for (int g = 0; g < G; ++g) all.insert(all.end(), ks[g]->len.begin(), ks[g]->len.end());
  return os_candidates_for(c, all, max_os, ks[0]->real);
}

}  // namespace

void autotune_impl(rf_ctx* c, int32_t G, const void* const* z_refs, rf_kernels* const* ks, int64_t W,
                   int32_t flags, int32_t max_os, rf_tune_entry* out, int32_t max_out, int32_t* n_out,
                   cudaStream_t s) {
  int64_t rows = 0, taps = 0;
  int32_t max_len = 0;
  for (int g = 0; g < G; ++g) {
    rows += ks[g]->k;
    taps += ks[g]->offset[ks[g]->k];
    max_len = std::max(max_len, ks[g]->max_len);
  }
  const double mean_len = rows ? (double)taps / (double)rows : 0.0;
  std::vector<Cand> cands;
  const bool f32 = c->g.dtype == RF_F32;
  if (f32 && c->n >= 512) cands = os_candidates(c, G, ks, std::max(1, max_os));
  // the tensor-core form costs 8 L flops per output times the split products, so it is timed
  // only for short kernels (mean length <= 4096 taps)
  // both tile layouts: 16-neighbour groups with stacked output tiles, and the widest groups
  if ((flags & RF_TUNE_ALLOW_SPLIT) && max_len <= gemm_max_len() && c->n % 128 == 0 && mean_len <= 4096.0) {
    cands.push_back(Cand{RF_ALGO_GEMM, 16, gemm_stacked_shifts(RF_PREC_BF16X6), RF_PREC_BF16X6, 0.0});
    cands.push_back(Cand{RF_ALGO_GEMM, gemm_wide_nj(RF_PREC_BF16X6), 1, RF_PREC_BF16X6, 0.0});
  }
  if (!f32 || max_len <= 1024) cands.push_back(Cand{RF_ALGO_DIRECT, 0, 0, RF_PREC_NATIVE, 0.0});
  RF_REQUIRE(!cands.empty(), "no reconstruction form to tune");
  const int64_t nw = (c->n + W - 1) / W;
  DevBuf pk, ak;
  pk.ensure(sizeof(float) * (size_t)std::max<int64_t>(1, rows * nw));
  ak.ensure(sizeof(int32_t) * (size_t)std::max<int64_t>(1, rows * nw));
  cudaEvent_t e0, e1;
  RF_CUDA(cudaEventCreate(&e0));
  RF_CUDA(cudaEventCreate(&e1));
  auto run = [&](const Cand& cd) {
    if ((cd.algo == RF_ALGO_OS || cd.algo == RF_ALGO_OS_BINS || cd.cut) && G > 1) {  // bucketed: batched
      reconstruct_batched(c, G, z_refs, ks, W, pk.as<float>(), ak.as<int32_t>(), s);
      return;
    }
    int64_t row = 0;
    for (int g = 0; g < G; ++g) {
      rf_kernels* k = ks[g];
      if (k->k) {
        float* mo = pk.as<float>() + row * nw;
        int32_t* ao = ak.as<int32_t>() + row * nw;
        if (cd.algo == RF_ALGO_OS || cd.algo == RF_ALGO_OS_BINS || cd.cut)
          reconstruct_os(c, z_refs[g], k, nullptr, W, mo, ao, s);
        else if (cd.algo == RF_ALGO_GEMM) reconstruct_gemm(c, z_refs[g], k, cd.prec, nullptr, W, mo, ao, s);
        else reconstruct_direct(c, z_refs[g], k, nullptr, W, mo, ao, s);
      }
      row += k->k;
    }
  };
  auto prepare = [&](const Cand& cd) {
    if (cd.cut) {  // two or three buckets: (algo, prec, block, part) below the cut, then the others
      const BucketSpec spec[3] = {BucketSpec{0, cd.algo, cd.prec, cd.block, cd.part},
                                  BucketSpec{cd.cut, cd.algo2, RF_PREC_NATIVE, cd.block2, cd.part2},
                                  BucketSpec{cd.cut3, cd.algo3, RF_PREC_NATIVE, cd.block3, cd.part3}};
      for (int g = 0; g < G; ++g) os_prepare_forms(c, ks[g], cd.cut3 ? 3 : 2, spec, s);
    } else if (cd.algo == RF_ALGO_OS_BINS) {
      const BucketSpec spec = BucketSpec{0, RF_ALGO_OS_BINS, RF_PREC_NATIVE, cd.block, cd.part};
      for (int g = 0; g < G; ++g) os_prepare_forms(c, ks[g], 1, &spec, s);
    } else if (cd.algo == RF_ALGO_OS) {
      for (int g = 0; g < G; ++g) os_prepare(c, ks[g], cd.block, cd.part, s);
    } else if (cd.algo == RF_ALGO_GEMM) {
      for (int g = 0; g < G; ++g) {
        ks[g]->gemm_pref_nj = cd.block;
        ks[g]->gemm_pref_s = cd.part;
      }
    }
  };
  auto time_cand = [&](const Cand& cd) {
    prepare(cd);
    run(cd);  // warm-up (and the tensor-core operand preparation)
    float best = 0.f;
    for (int r = 0; r < 3; ++r) {
      RF_CUDA(cudaEventRecord(e0, s));
      run(cd);
      RF_CUDA(cudaEventRecord(e1, s));
      RF_CUDA(cudaEventSynchronize(e1));
      float t = 0.f;
      RF_CUDA(cudaEventElapsedTime(&t, e0, e1));
      best = r == 0 ? t : std::min(best, t);
    }
    return best;
  };
  std::vector<float> ms;
  for (const Cand& cd : cands) ms.push_back(time_cand(cd));
  // two-bucket variants around the fastest single layout: the kernels below a cut run with
  // one of the two layouts of least modelled cost for them
  if (f32 && c->n >= 512 && max_os > 0) {
    size_t best_os = cands.size();
    for (size_t i = 0; i < cands.size(); ++i)
      if (cands[i].algo == RF_ALGO_OS && (best_os == cands.size() || ms[i] < ms[best_os])) best_os = i;
    if (best_os < cands.size()) {
      const Cand lead = cands[best_os];
      std::vector<Cand> extra;
      for (const int cut : {2048, 4096, 8192}) {
        std::vector<int> shortL;
        bool any_long = false;
        for (int g = 0; g < G; ++g)
          for (const int L : ks[g]->len) {
            if (L < cut) shortL.push_back(L);
            else any_long = true;
          }
        if (shortL.empty() || !any_long) continue;
        std::vector<Cand> sc = os_candidates_for(c, shortL, 2, ks[0]->real);
        for (Cand cd : sc) {
          if (cd.block == lead.block && cd.part == lead.part) continue;
          cd.cut = cut;
          cd.block2 = lead.block;
          cd.part2 = lead.part;
          extra.push_back(cd);
        }
      }
      // mixed forms: the tensor-core form (bf16x6, the library's tile rule) for the shortest
      // kernels (about an eighth of them, at most 4096 taps), the fastest layout above
      if ((flags & RF_TUNE_ALLOW_SPLIT) && c->n % 128 == 0) {
        std::vector<int> all;
        for (int g = 0; g < G; ++g) all.insert(all.end(), ks[g]->len.begin(), ks[g]->len.end());
        std::sort(all.begin(), all.end());
        if (all.size() >= 8) {
          int cut = 256;
          while (cut < 4096 && cut <= all[all.size() / 8]) cut *= 2;
          const bool some_short = all.front() < cut, some_long = all.back() >= cut;
          if (some_short && some_long) {
            Cand cd{RF_ALGO_GEMM, 0, 0, RF_PREC_BF16X6, 0.0};
            cd.cut = cut;
            cd.block2 = lead.block;
            cd.part2 = lead.part;
            extra.push_back(cd);
          }
        }
      }
      // two-phase overlap-save (partition sums per bin) for the long kernels: the fastest single
      // layout in that form, and every two-bucket candidate so far with its upper bucket so
      if (bins_layout_ok(lead.block, lead.part)) {
        Cand one{RF_ALGO_OS_BINS, lead.block, lead.part, RF_PREC_NATIVE, 0.0};
        extra.push_back(one);
      }
      // ... and three buckets: the two-phase form only for the kernels of many partitions (at
      // least 4, 8 or 16), where its per-bin sums pay for the buffer round trip
      // The two-phase form also runs 32768-point blocks on CTA pairs (Lp = 16384: half the
      // partitions of Lp = 8192, so half the per-bin multiply-adds, for a block tail on two SMs).
      std::vector<Cand> twos;
      int32_t lmax = 0;
      for (int g = 0; g < G; ++g) lmax = std::max(lmax, ks[g]->max_len);
      const bool pair_ok = !ks[0]->real && c->n >= 32768;
      for (const Cand& cd : extra)
        if (cd.cut && cd.algo == RF_ALGO_OS && cd.algo2 == RF_ALGO_OS && bins_layout_ok(cd.block2, cd.part2)) {
          Cand t = cd;
          t.algo2 = RF_ALGO_OS_BINS;
          twos.push_back(t);
          for (const int np : {4, 8, 16}) {
            const int cut3 = np * cd.part2;
            if (cut3 <= cd.cut || cut3 > lmax) continue;
            Cand three = cd;
            three.cut3 = cut3;
            three.block3 = cd.block2;
            three.part3 = cd.part2;
            three.algo3 = RF_ALGO_OS_BINS;
            twos.push_back(three);
            if (pair_ok && cd.block2 == 16384) {
              three.block3 = 32768;
              three.part3 = 16384;
              twos.push_back(three);
            }
          }
        }
      extra.insert(extra.end(), twos.begin(), twos.end());
      for (const Cand& cd : extra) {
        cands.push_back(cd);
        ms.push_back(time_cand(cd));
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  size_t win = 0;
  for (size_t i = 1; i < cands.size(); ++i)
    if (ms[i] < ms[win]) win = i;
  const Cand& w = cands[win];
  prepare(w);
  for (int g = 0; g < G; ++g) {
    // bucketed preparations (overlap-save, two-phase or mixed) run through the overlap-save entry
    const bool bucketed = w.cut || w.algo == RF_ALGO_OS_BINS;
    ks[g]->tuned_algo = bucketed ? RF_ALGO_OS : w.algo;
    ks[g]->tuned_prec = bucketed ? RF_PREC_NATIVE : w.prec;
  }
  RF_CUDA(cudaStreamSynchronize(s));
  // the winner first, then the others in the order they were timed
  int32_t n = 0;
  auto put = [&](size_t i) {
    const Cand& cd = cands[i];
    if (n < max_out && out)
      out[n] = rf_tune_entry{cd.algo,  cd.block,  cd.part,  cd.prec,  cd.cut,  cd.block2,
                             cd.part2, cd.cut ? cd.algo2 : 0,     cd.cut3, cd.block3, cd.part3,
                             cd.cut3 ? cd.algo3 : 0,               ms[i]};
    ++n;
  };
  put(win);
  for (size_t i = 0; i < cands.size(); ++i)
    if (i != win) put(i);
  if (n_out) *n_out = std::min(n, max_out);
}

}  // namespace rf
