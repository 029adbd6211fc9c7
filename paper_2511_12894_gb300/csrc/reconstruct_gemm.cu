// Direct reconstruction (Eq. 8) as a complex GEMM on the tcgen05 tensor cores, with
// split-BF16 operands and FP32 accumulation in tensor memory.
//
// For a tile of 128 outputs i' = i0 + m and a group of NJ neighbours whose taps are padded
// to LP (a multiple of 16), with taps read in reverse (t = LP - 1 - l):
//   w_j[i0 + m] = sum_t z[b + m + t] c_j[LP - 1 - t],   b = i0 - LP + 1,
// a Hankel matrix A[m][t] = z[b + m + t] times the tap matrix.  Real and imaginary planes
// give two real products per output column pair (re, im):
//   D[m][2j]   = sum_t zr A_t cr_j - zi A_t ci_j,    D[m][2j+1] = sum_t zr ci_j + zi cr_j,
// i.e. D = A_r B_r + A_i B_i with B_r = [cr ci], B_i = [-ci cr] per neighbour.
//
// The Hankel operand is never expanded in shared memory: in the no-swizzle K-major layout an
// 8x8 BF16 core matrix (8 rows of 16 bytes) at row block r and K block q holds
// z[b + 8(r + q) + a + e] (a, e < 8), which depends on r + q only.  Shared memory keeps the
// distinct core matrices H_d, d = r + q, back to back, and the descriptor uses the same
// 128-byte stride for the M and K directions.  Global memory holds every core matrix as a
// 128-byte record per start position, so a chunk's H_d arrive by one TMA box.
//
// Split precision: x = x0 + x1 + x2 with x_k = bf16(x - x0 - ... - x_{k-1}); the products
// kept are (0,0) for BF16, + (0,1),(1,0) for x3, + (0,2),(1,1),(2,0) for x6, + (1,2),(2,1),(2,2)
// for x9.  The tensor core's FP32 accumulation loses a fraction of an ulp of the running
// sum at every MMA, so the products of every K chunk (at most 128 taps) accumulate in tensor
// memory by order (ta + tb) and the block adds them into FP32 register sums (round to
// nearest), corrections apart from the leading product.
//
// 3xTF32 runs the same tiles with kind::tf32 MMAs: x = x0 + x1, x0 = tf32(x) and
// x1 = tf32(x - x0) (each TF32 term carries 11 significant bits, so x1 resolves x to about
// 2^-22), products (0,0), (0,1), (1,0).  A TF32 core matrix row is 16 bytes = 4 values and
// an MMA spans K = 8, so the Hankel core matrix at row block r and K block q starts at
// z[b + 8r + 4q], i.e. depends on d = 2r + q: consecutive d are the K neighbours and d + 2
// the next row block.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <memory>

#include "cplx.cuh"
#include "rf_internal.h"

namespace rf {

namespace {

constexpr int kGemmThreads = 128;
constexpr int kGemmM = 128;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor: no swizzle, K-major, relative offsets.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor: FP32 D, K-major A and B of format fmt (kind::f16: 1 = BF16;
// kind::tf32: 2 = TF32), M = 128, N.
__host__ __device__ constexpr uint32_t mma_idesc(int N, uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kGemmM >> 4) << 24);
}

// Operand format of a split precision: TF32 terms are 4-byte words (core-matrix rows of 4
// values, K = 8 per MMA), BF16 terms 2-byte (rows of 8 values, K = 16 per MMA).
__host__ __device__ constexpr bool prec_tf32(int prec) { return prec == RF_PREC_3XTF32; }
__host__ __device__ constexpr int prec_ebytes(int prec) { return prec_tf32(prec) ? 4 : 2; }
// distinct Hankel core matrices of a K chunk of KC taps (d = r + q, or 2r + q for TF32)
__host__ __device__ constexpr int hankel_cores(int prec, int KC) {
  return prec_tf32(prec) ? 30 + KC / 4 : 15 + KC / 8;
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

template <typename R>
__device__ __forceinline__ void split3(R v, __nv_bfloat16& s0, __nv_bfloat16& s1, __nv_bfloat16& s2) {
  s0 = __float2bfloat16_rn((float)v);
  const R r1 = v - (R)__bfloat162float(s0);
  s1 = __float2bfloat16_rn((float)r1);
  const R r2 = r1 - (R)__bfloat162float(s1);
  s2 = __float2bfloat16_rn((float)r2);
}

template <typename R>
__device__ __forceinline__ void split2_tf32(R v, float& s0, float& s1) {
  s0 = tf32_rna((float)v);
  s1 = tf32_rna((float)(v - (R)s0));
}

// Product pairs (A term, B term) of each precision, in issue order.
__host__ __device__ constexpr int prec_products(int prec) {
  return prec == RF_PREC_BF16 ? 1 : (prec == RF_PREC_BF16X3 || prec == RF_PREC_3XTF32) ? 3 : prec == RF_PREC_BF16X6 ? 6 : 9;
}
__host__ __device__ constexpr int prec_terms(int prec) {
  return prec == RF_PREC_BF16 ? 1 : (prec == RF_PREC_BF16X3 || prec == RF_PREC_3XTF32) ? 2 : 3;
}

// Tap operands of one neighbour group, prepared once per kernel set, chunk by chunk:
// [K chunk c][plane (r, i)][term][NC/8 row blocks][KC/8 K blocks][8 rows][8 BF16] (TF32:
// [KC/4 K blocks][8 rows][4 words]) over the extended K range t in [0, NCK KC), NCK KC =
// LP + 128 (S - 1).  Column s 2 NJ + 2j (+1) = re (im) of neighbour j of the group at output
// shift s, holding tap l = LP - 1 - t + 128 s (zero outside the kernel); plane r holds
// (cr, ci), plane i holds (-ci, cr).
template <typename V>
__global__ void k_gemm_prep_b(const void* __restrict__ taps_v, bool real_taps, const int64_t* __restrict__ off,
                              const int* __restrict__ len, int k, int NJ, int S, int KC, int NCK, int LP, int terms,
                              bool tf32, void* __restrict__ out_v) {
  using R = typename real_of<V>::type;
  const int g = blockIdx.y;
  const int NC = S * 2 * NJ;
  const int LPX = KC * NCK;
  const int64_t per_plane_term = (int64_t)NC * KC;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)NC * LPX;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(e / LPX), t = (int)(e % LPX);
    const int c = t / KC, tl = t % KC;
    const int sh = col / (2 * NJ);
    const int j = g * NJ + (col % (2 * NJ)) / 2;
    R cr = 0, ci = 0;
    if (j < k) {
      const int l = LP - 1 - t + kGemmM * sh;
      if (l >= 0 && l < len[j]) {
        if (real_taps) {  // real-form set: real taps, imaginary parts zero
          cr = static_cast<const R*>(taps_v)[off[j] + l];
        } else {
          const V v = static_cast<const V*>(taps_v)[off[j] + l];
          cr = v.x;
          ci = v.y;
        }
      }
    }
    const R vr = (col & 1) ? ci : cr;
    const R vi = (col & 1) ? cr : -ci;
    const int64_t chunk = ((int64_t)g * NCK + c) * 2 * terms * per_plane_term;
    if (tf32) {
      float rr[2], ii[2];
      split2_tf32<R>(vr, rr[0], rr[1]);
      split2_tf32<R>(vi, ii[0], ii[1]);
      float* oc = static_cast<float*>(out_v) + chunk;
      const int64_t pos = (int64_t)(col / 8) * (KC / 4) * 32 + (tl / 4) * 32 + (col % 8) * 4 + (tl % 4);
      for (int s = 0; s < terms; ++s) {
        oc[(0 * terms + s) * per_plane_term + pos] = rr[s];
        oc[(1 * terms + s) * per_plane_term + pos] = ii[s];
      }
    } else {
      __nv_bfloat16 rr[3], ii[3];
      split3<R>(vr, rr[0], rr[1], rr[2]);
      split3<R>(vi, ii[0], ii[1], ii[2]);
      __nv_bfloat16* oc = static_cast<__nv_bfloat16*>(out_v) + chunk;
      const int64_t pos = (int64_t)(col / 8) * (KC / 8) * 64 + (tl / 8) * 64 + (col % 8) * 8 + (tl % 8);
      for (int s = 0; s < terms; ++s) {
        oc[(0 * terms + s) * per_plane_term + pos] = rr[s];
        oc[(1 * terms + s) * per_plane_term + pos] = ii[s];
      }
    }
  }
}

// z_ref split into BF16 (or TF32) terms once per call and stored as the Hankel core matrices the
// MMAs read, for every start position: record [pt][d] (pt = plane r/i x term s) is the 8 x 16-byte
// core matrix whose row a holds term s of elements x = R d + a + e - pad (e < R values per row;
// R = 8 BF16 or 4 TF32) of the circular sequence, so a chunk's distinct core matrices are one
// contiguous run of records per (plane, term) and one TMA box loads them all.  pad = 7 (mod 8)
// makes every chunk start a whole record; the tail covers the extended K range of up to 8 output
// shifts.  The split runs in FP32 (complex128 inputs are rounded to FP32 first, well inside the
// resolution of the split terms).
static int64_t gemm_zpad(int64_t LP) { return ((LP + 8 + 7) / 8) * 8 + 7; }
static int64_t gemm_zlen(int64_t n, int64_t LP) { return ((gemm_zpad(LP) + n + 1024 + 160 + 7) / 8) * 8; }
static int64_t gemm_zrecs(int64_t n, int64_t LP, bool tf32) { return gemm_zlen(n, LP) / (tf32 ? 4 : 8); }

__device__ __forceinline__ uint4 pack8(const __nv_bfloat16 (&v)[8]) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
    w[i] = (uint32_t)__bfloat16_as_ushort(v[2 * i]) | ((uint32_t)__bfloat16_as_ushort(v[2 * i + 1]) << 16);
  return make_uint4(w[0], w[1], w[2], w[3]);
}

template <typename V>
__global__ void k_gemm_split_z(const V* __restrict__ z, int64_t n, int64_t pad, int64_t recs, int terms,
                               __nv_bfloat16* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // (record d, row a)
  if (t >= recs * 8) return;
  const int64_t d = t >> 3;
  const int a = (int)(t & 7);
  __nv_bfloat16 r[3][8], im[3][8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const V v = z[(8 * d + a + e - pad) & (n - 1)];
    split3<float>((float)v.x, r[0][e], r[1][e], r[2][e]);
    split3<float>((float)v.y, im[0][e], im[1][e], im[2][e]);
  }
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    if (s < terms) {
      *reinterpret_cast<uint4*>(out + ((int64_t)(0 * terms + s) * recs + d) * 64 + a * 8) = pack8(r[s]);
      *reinterpret_cast<uint4*>(out + ((int64_t)(1 * terms + s) * recs + d) * 64 + a * 8) = pack8(im[s]);
    }
  }
}

template <typename V>
__global__ void k_gemm_split_z_tf32(const V* __restrict__ z, int64_t n, int64_t pad, int64_t recs,
                                    float* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // (record d, row a)
  if (t >= recs * 8) return;
  const int64_t d = t >> 3;
  const int a = (int)(t & 7);
  float r[2][4], im[2][4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const V v = z[(4 * d + a + e - pad) & (n - 1)];
    split2_tf32<float>((float)v.x, r[0][e], r[1][e]);
    split2_tf32<float>((float)v.y, im[0][e], im[1][e]);
  }
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    *reinterpret_cast<float4*>(out + ((int64_t)(0 * 2 + s) * recs + d) * 32 + a * 4) =
        make_float4(r[s][0], r[s][1], r[s][2], r[s][3]);
    *reinterpret_cast<float4*>(out + ((int64_t)(1 * 2 + s) * recs + d) * 32 + a * 4) =
        make_float4(im[s][0], im[s][1], im[s][2], im[s][3]);
  }
}

__device__ __forceinline__ unsigned long long gemm_key(float v, unsigned int i) {
  return ((unsigned long long)__float_as_uint(v) << 32) | (unsigned long long)(0xffffffffu - i);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// Bounded wait for phase `phase` of an mbarrier; true when it completed.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar_addr, uint32_t phase, int limit = 1 << 24) {
  uint32_t done = 0;
  for (int it = 0; it < limit && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done) : "r"(mbar_addr), "r"(phase) : "memory");
  }
  return done != 0;
}

// B terms multiplied with A term ta: x9 keeps all three, the others the terms tb <= TERMS-1-ta.
__host__ __device__ constexpr int b_terms_for(int prec, int ta) {
  return prec == RF_PREC_BF16X9 ? 3 : prec_terms(prec) - ta;
}
// Tensor-memory column groups.  The products of one order ta + tb accumulate into one group
// of NC columns (the leading product alone, then the first-order corrections, ...): the MMA of
// A term ta covers B terms 0.., so it writes orders ta, ta + 1, ... and starts at group ta, and
// the MMA of A term 0 reaches every order first, so it initialises them all.  bf16x9's orders
// 3 and 4 are first reached by later A terms, so it keeps one group per product.
__host__ __device__ constexpr bool prec_merged(int prec) { return prec != RF_PREC_BF16X9; }
__host__ __device__ constexpr int prec_groups(int prec) {
  return prec_merged(prec) ? prec_terms(prec) : prec_products(prec);
}
__host__ __device__ constexpr int tile_col(int prec, int ta, int NC) {
  if (prec_merged(prec)) return ta * NC;
  int c = 0;
  for (int t = 0; t < ta; ++t) c += NC * b_terms_for(prec, t);
  return c;
}
// Output shifts stacked along N for a group of NJ neighbours: the widest power of two S <= 8
// whose MMA of A term 0 (S * 2 NJ columns per B term) stays within N = 256 and whose column
// groups fit the 512 columns of tensor memory.
__host__ __device__ constexpr int gemm_shifts_max(int prec, int NJ) {
  int s = 8;
  while (s > 1 && (s * 2 * NJ * b_terms_for(prec, 0) > 256 || s * 2 * NJ * prec_groups(prec) > 512)) s /= 2;
  return s;
}

// One block: TM consecutive super-tiles of S x 128 outputs of one group of NJ neighbours.
// Output shift s (tile rows i0 + 128 s + m) needs z[b + m + t'] at t' = t + 128 s, so all S
// tiles share the Hankel operand of an extended K range (LP + 128 (S - 1) taps) and the tap
// operand holds, per shift, the taps moved down by 128 s (zero outside the kernel): one MMA
// serves S tiles, NC = S x 2 NJ columns per B term.  The (tile, chunk) steps q of the block run
// through two shared-memory stages: thread 0 loads step q + 1 (the chunk's Hankel core matrices
// by one TMA box, its tap operands by one bulk copy, both completing on full[stage]) while the
// MMAs of step q run; it issues one MMA per (K step, plane, A term) whose N spans every B term
// paired with that A term; the block folds the chunk's column groups into FP32 register sums
// (plain BF16 accumulates in tensor memory) and after the tile's last chunk writes the outputs
// or their window peaks.
template <typename V, int NJ, int PREC, bool WINMAX, int S>
__global__ void __launch_bounds__(kGemmThreads, 1) k_gemm(const __grid_constant__ CUtensorMap zmap, int64_t zpad,
                                                          int64_t n, const void* __restrict__ Bg, int KC, int NCK,
                                                          int LP, int k, const int* __restrict__ lag0, int TM,
                                                          V* __restrict__ z_out, unsigned long long* __restrict__ keys,
                                                          int64_t W, int64_t nw, int tmem_cols,
                                                          int* __restrict__ status) {
  using R = typename real_of<V>::type;
  constexpr int NC = S * 2 * NJ;           // columns per B term (all shifts)
  constexpr int TERMS = prec_terms(PREC);
  constexpr bool FOLD = PREC != RF_PREC_BF16;
  constexpr bool MERGED = prec_merged(PREC);
  constexpr bool TF = prec_tf32(PREC);
  constexpr int EB = prec_ebytes(PREC);     // bytes per operand value
  constexpr int RSTEP = TF ? 4 : 8;         // elements between consecutive core-matrix records
  static_assert(NC % 16 == 0 && NC * b_terms_for(PREC, 0) <= 256, "MMA width");
  static_assert((2 * NJ) % 16 == 0, "a 16-column slice holds one shift");
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) unsigned long long mbar, full[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = blockIdx.y;
  const int nH = hankel_cores(PREC, KC);              // distinct Hankel core matrices per chunk
  const int a_bytes = nH * 128;                       // per (plane, term)
  const int b_bytes = NC * KC * EB;                   // per (plane, term)
  const uint32_t a_stage = (uint32_t)(2 * TERMS * a_bytes), b_stage = (uint32_t)(2 * TERMS * b_bytes);
  // stage st: [plane][term][nH][128 B] Hankel cores, then [plane][term][NC/8][KC/(16/EB)][128 B] taps
  auto stage_a = [&](int st) { return smem + st * (a_stage + b_stage); };
  const int64_t mask = n - 1;
  const unsigned char* Bgrp = static_cast<const unsigned char*>(Bg) + (int64_t)g * NCK * b_stage;
  const int64_t tiles = (n + kGemmM * S - 1) / (kGemmM * S);
  const int64_t tile0 = (int64_t)blockIdx.x * TM;
  const int my_tiles = (int)max((int64_t)0, min((int64_t)TM, tiles - tile0));
  const int Q = my_tiles * NCK;                       // (tile, chunk) steps of this block

  // thread 0: start the loads of step q into stage st
  auto issue_loads = [&](int q, int st) {
    const int tile = q / NCK, c = q - tile * NCK;
    const int64_t i0 = (tile0 + tile) * (kGemmM * S);
    const int64_t bc = i0 - LP + 1 + (int64_t)c * KC + zpad;  // first element of the chunk (a record start)
    const uint32_t fb = smem_u32(&full[st]);
    unsigned char* sa = stage_a(st);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(a_stage + b_stage)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(sa)),
        "l"(reinterpret_cast<uint64_t>(&zmap)), "r"(0), "r"((int)(bc / RSTEP)), "r"(0), "r"(fb)
        : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(sa + a_stage)),
        "l"(Bgrp + (int64_t)c * b_stage), "r"(b_stage), "r"(fb)
        : "memory");
  };

  if (tid == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&zmap)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t mbar_addr = smem_u32(&mbar);
  uint32_t phase = 0;
  const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
  const unsigned int Wu = (unsigned int)(W < n ? W : n), nwu = (unsigned int)nw;  // n <= 2^24
  if (tid == 0 && Q > 0) issue_loads(0, 0);
  float run[FOLD ? NC : 1];

  for (int q = 0; q < Q; ++q) {
    const int st = q & 1, tile = q / NCK, c = q - tile * NCK;
    const int64_t i0 = (tile0 + tile) * (kGemmM * S);
    if (c == 0) {
#pragma unroll
      for (int cidx = 0; cidx < (FOLD ? NC : 1); ++cidx) run[cidx] = 0.f;
    }
    bool lok = true, next = false;
    if (tid == 0) {
      // the other stage was last read by the MMAs of step q - 1, which have completed: its
      // next loads start before this step's MMAs, a whole step ahead of their use
      if (q + 1 < Q) {
        issue_loads(q + 1, st ^ 1);
        next = true;
      }
      lok = mbar_wait(smem_u32(&full[st]), (uint32_t)((q >> 1) & 1));
      if (lok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        unsigned char* sa = stage_a(st);
        // A K step (32 bytes of every row: K = 16 BF16 or 8 TF32 values) spans two core
        // matrices along K, so step ks adds ks * 256 bytes to each start address, i.e. ks * 16
        // to the descriptor's low field (addresses stay below 256 KB, so the field never
        // carries).  Leading byte offset = next core matrix along K, stride byte offset = next
        // 8-row block along M or N.
        uint64_t adesc[2 * TERMS], bdesc[2];
#pragma unroll
        for (int i = 0; i < 2 * TERMS; ++i) adesc[i] = smem_desc(smem_u32(sa + i * a_bytes), 128, TF ? 256 : 128);
#pragma unroll
        for (int pl = 0; pl < 2; ++pl)
          bdesc[pl] = smem_desc(smem_u32(sa + a_stage + pl * TERMS * b_bytes), 128, KC * 8 * EB);
        for (int ks = 0; ks < KC * EB / 32; ++ks) {
          const uint64_t koff = (uint64_t)(ks * 16);
#pragma unroll
          for (int pl = 0; pl < 2; ++pl)
#pragma unroll
            for (int ta = 0; ta < TERMS; ++ta) {
              const uint32_t idesc = mma_idesc(NC * b_terms_for(PREC, ta), TF ? 2u : 1u);
              const uint32_t d = tmem + (uint32_t)tile_col(PREC, ta, NC);
              // the first MMA of a chunk (of the tile, for plain BF16) overwrites its columns;
              // merged groups are all first written by A term 0
              const bool first = (FOLD || c == 0) && ks == 0 && pl == 0 && (!MERGED || ta == 0);
              const uint32_t acc = first ? 0u : 1u;
              if constexpr (TF)
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                    "l"(adesc[pl * TERMS + ta] + koff), "l"(bdesc[pl] + koff), "r"(idesc), "r"(acc));
              else
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                    "l"(adesc[pl * TERMS + ta] + koff), "l"(bdesc[pl] + koff), "r"(idesc), "r"(acc));
            }
        }
      }
      // the commit arrives once every MMA issued so far has completed (at once when none was)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_addr)
                   : "memory");
    }
    const bool done = mbar_wait(mbar_addr, phase);
    phase ^= 1u;
    if (!__syncthreads_and(done && lok)) {
      if (tid == 0) {
        atomicExch(status, (int)RF_ETIMEOUT);
        // bounded waits for whatever is still in flight before shared and tensor memory go
        if (!lok) mbar_wait(smem_u32(&full[st]), (uint32_t)((q >> 1) & 1));
        if (next) mbar_wait(smem_u32(&full[st ^ 1]), (uint32_t)(((q + 1) >> 1) & 1));
        if (!done) mbar_wait(mbar_addr, phase ^ 1u);
      }
      __syncthreads();
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if constexpr (FOLD) {
      // row sums of the chunk: the leading product plus the corrections
      constexpr int NG = prec_groups(PREC);
#pragma unroll
      for (int h = 0; h < NC / 16; ++h) {
        float big[16], small[16];
#pragma unroll
        for (int g0 = 0; g0 < NG; g0 += 3) {  // up to three loads in flight per wait
          uint32_t v[3][16];
#pragma unroll
          for (int gg = 0; gg < 3; ++gg)
            if (g0 + gg < NG) tmem_ld16(taddr + (uint32_t)((g0 + gg) * NC + 16 * h), v[gg]);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int gg = 0; gg < 3; ++gg)
#pragma unroll
            for (int cc = 0; cc < 16; ++cc) {
              if (g0 + gg == 0) {
                big[cc] = __uint_as_float(v[gg][cc]);
                small[cc] = 0.f;
              } else if (g0 + gg < NG) {
                small[cc] += __uint_as_float(v[gg][cc]);
              }
            }
        }
#pragma unroll
        for (int cc = 0; cc < 16; ++cc) run[16 * h + cc] += big[cc] + small[cc];
      }
    }
    if (c == NCK - 1) {
#pragma unroll
      for (int h = 0; h < NC / 16; ++h) {
        const int sh = (16 * h) / (2 * NJ);             // output shift of this column slice
        if (i0 + (int64_t)kGemmM * sh >= n) break;      // uniform across the block
        const int64_t ip = i0 + kGemmM * sh + warp * 32 + lane;  // i'
        const int jb = ((16 * h) % (2 * NJ)) / 2;       // first neighbour of the slice
        float val[16];
        if constexpr (FOLD) {
#pragma unroll
          for (int cc = 0; cc < 16; ++cc) val[cc] = run[16 * h + cc];
        } else {
          uint32_t v[16];
          tmem_ld16(taddr + (uint32_t)(16 * h), v);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int cc = 0; cc < 16; ++cc) val[cc] = __uint_as_float(v[cc]);
        }
        const int nj = min(8, k - (g * NJ + jb));  // neighbours in this slice (uniform)
        if (nj <= 0) continue;
        if constexpr (!WINMAX) {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            if (jj >= nj) break;
            const int j = g * NJ + jb + jj;
            const unsigned int i = (unsigned int)((ip + lag0[j]) & mask);
            z_out[(int64_t)j * n + i] = cmake<V>((R)val[2 * jj], (R)val[2 * jj + 1]);
          }
        } else {
          // The warp's 32 outputs are consecutive modulo n: usually they fall in lane 0's window
          // wA and the next one wB (window 0 after the wrap), decided by comparison; per window
          // the largest |z|^2 (non-negative floats order as their bit patterns) and then the
          // smallest index holding it come from two 32-bit warp reductions.  The slice's
          // neighbours are independent chains, interleaved.
          unsigned int iv[8], pb[8], wA[8], wB[8];
          bool inA[8], inB[8], slow = false;
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const int j = g * NJ + jb + min(jj, nj - 1);
            iv[jj] = (unsigned int)((ip + lag0[j]) & mask);
            pb[jj] = __float_as_uint(val[2 * jj] * val[2 * jj] + val[2 * jj + 1] * val[2 * jj + 1]);
            wA[jj] = (unsigned int)((ip - lane + lag0[j]) & mask) / Wu;  // lane 0's window
            wB[jj] = (wA[jj] + 1 == nwu) ? 0u : wA[jj] + 1;
            inA[jj] = iv[jj] - wA[jj] * Wu < Wu;
            inB[jj] = !inA[jj] && iv[jj] - wB[jj] * Wu < Wu;
            if (jj < nj) slow |= !(inA[jj] || inB[jj]);
          }
          if (__any_sync(0xffffffffu, slow)) {
#pragma unroll
            for (int jj = 0; jj < 8; ++jj)
              if (jj < nj)
                atomicMax(keys + (int64_t)(g * NJ + jb + jj) * nw + iv[jj] / Wu,
                          gemm_key(__uint_as_float(pb[jj]), iv[jj]));
          } else {
            unsigned int mA[8], mB[8], xA[8], xB[8];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
              mA[jj] = __reduce_max_sync(0xffffffffu, inA[jj] ? pb[jj] : 0u);
              mB[jj] = __reduce_max_sync(0xffffffffu, inB[jj] ? pb[jj] : 0u);
            }
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
              xA[jj] = __reduce_min_sync(0xffffffffu, (inA[jj] && pb[jj] == mA[jj]) ? iv[jj] : 0xffffffffu);
              xB[jj] = __reduce_min_sync(0xffffffffu, (inB[jj] && pb[jj] == mB[jj]) ? iv[jj] : 0xffffffffu);
            }
            if (lane == 0) {
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) {
                if (jj >= nj) break;
                unsigned long long* kj = keys + (int64_t)(g * NJ + jb + jj) * nw;
                if (xA[jj] != 0xffffffffu) atomicMax(kj + wA[jj], gemm_key(__uint_as_float(mA[jj]), xA[jj]));
                if (xB[jj] != 0xffffffffu) atomicMax(kj + wB[jj], gemm_key(__uint_as_float(mB[jj]), xB[jj]));
              }
            }
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // tensor memory is rewritten by the next step's MMAs
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

__global__ void k_gemm_unpack(const unsigned long long* __restrict__ keys, int64_t count, float* __restrict__ mx,
                              int* __restrict__ arg) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const unsigned long long kk = keys[i];
  mx[i] = __uint_as_float((unsigned int)(kk >> 32));
  arg[i] = (int)(0xffffffffu - (unsigned int)(kk & 0xffffffffull));
}

// Two stages of (Hankel records, tap operands).
size_t gemm_smem_bytes(int prec, int NJ, int S, int KC) {
  const int terms = prec_terms(prec);
  return 2 * ((size_t)2 * terms * hankel_cores(prec, KC) * 128 +
              (size_t)2 * terms * (S * 2 * NJ) * KC * prec_ebytes(prec)) +
         1024;
}

// Tensor map over the core-matrix records: element type BF16 (or 32-bit words for TF32),
// dims (values per record, records, planes x terms), no swizzle, zero fill outside.
CUtensorMap gemm_tensor_map(void* base, bool tf32, int64_t recs, int planes, int box_recs) {
  // looked up once per process; the initialisation of a function-local static is thread-safe
  // and is retried on the next call if it throws
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    cudaDriverEntryPointQueryResult q{};
    void* fn = nullptr;
    RF_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    RF_REQUIRE(fn != nullptr && q == cudaDriverEntryPointSuccess, "cuTensorMapEncodeTiled is not available");
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  const cuuint32_t per = tf32 ? 32 : 64;  // values per 128-byte record
  CUtensorMap m;
  const cuuint64_t dims[3] = {per, (cuuint64_t)recs, (cuuint64_t)planes};
  const cuuint64_t strides[2] = {128, (cuuint64_t)recs * 128};
  const cuuint32_t box[3] = {per, (cuuint32_t)box_recs, (cuuint32_t)planes};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = encode(&m, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base,
                            dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  RF_REQUIRE(r == CUDA_SUCCESS, "tensor map for the Hankel records rejected (CUresult %d)", (int)r);
  return m;
}

// Tensor-memory columns: one group of S x 2 NJ columns per product order (per product for
// bf16x9), rounded up to a power of two.
int gemm_tmem_cols(int prec, int NJ, int S) {
  const int need = prec_groups(prec) * S * 2 * NJ;
  int cols = 32;
  while (cols < need) cols *= 2;
  return cols;
}

// Neighbours per group: the widest MMA (all B terms of A term 0) must fit N <= 256, and the
// column groups must fit the 512 of tensor memory.
__host__ __device__ constexpr int gemm_nj_max(int prec) {
  return prec == RF_PREC_BF16                                 ? 128
         : (prec == RF_PREC_BF16X3 || prec == RF_PREC_3XTF32) ? 48
         : prec == RF_PREC_BF16X6                             ? 40
                                                              : 24;
}

template <typename V, int NJ, int PREC, bool WINMAX, int S>
void launch_gemm(rf_ctx* c, const rf_kernels* kern, const V* z_ref, V* z_out, unsigned long long* keys, int64_t W,
                 int64_t nw, cudaStream_t s) {
  const int KC = kern->gemm_KC, NCK = kern->gemm_NCK, LP = kern->gemm_LP;
  const int cols = gemm_tmem_cols(PREC, NJ, S);
  RF_REQUIRE(cols <= 512, "tensor-core form: %d tensor-memory columns needed", cols);
  // shared memory sized so that the blocks resident on one SM never ask for more than the
  // 512 tensor-memory columns of the SM (an allocation would otherwise wait for a release)
  const size_t smem_max = 227 * 1024;
  const int max_blocks = 512 / cols;
  size_t smem = gemm_smem_bytes(PREC, NJ, S, KC);
  smem = std::max(smem, smem_max / (size_t)(max_blocks + 1) + 1024);
  constexpr size_t smem_cap = 220 * 1024;
  smem = std::min(smem, smem_cap);
  auto fn = k_gemm<V, NJ, PREC, WINMAX, S>;
  // The dynamic shared-memory limit is a process-wide attribute of the function, so it is set to
  // the cap that bounds every launch: a context on another host thread never lowers it under a
  // launch of this one.  The tensor-memory occupancy check runs once per (device, size).
  static std::atomic<size_t> checked[16];
  const int dv = c->device & 15;
  if (checked[dv].load(std::memory_order_acquire) != smem) {
    RF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cap));
    int per_sm = 0;
    RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kGemmThreads, smem));
    RF_REQUIRE(per_sm >= 1 && per_sm * cols <= 512,
               "tensor-core form: %d blocks per SM x %d columns exceed tensor memory", per_sm, cols);
    checked[dv].store(smem, std::memory_order_release);
  }
  const int64_t tiles = (c->n + kGemmM * S - 1) / (kGemmM * S);
  const int groups = (kern->k + NJ - 1) / NJ;
  int TM = 1;
  while (TM < 16 && (tiles / (TM * 2)) * groups >= 4LL * c->nsm) TM *= 2;
  dim3 grid((unsigned)((tiles + TM - 1) / TM), (unsigned)groups);
  // z_ref split into BF16 (TF32) core-matrix records, padded so that no Hankel window wraps
  constexpr bool TF = prec_tf32(PREC);
  const int64_t zpad = gemm_zpad(LP), recs = gemm_zrecs(c->n, LP, TF);
  c->scratch2.ensure(gemm_zplanes_bytes(c->n, LP, PREC));
  void* zp = c->scratch2.as<unsigned char>();
  const unsigned split_blocks = (unsigned)((recs * 8 + 255) / 256);
  if constexpr (TF)
    k_gemm_split_z_tf32<V><<<split_blocks, 256, 0, s>>>(z_ref, c->n, zpad, recs, static_cast<float*>(zp));
  else
    k_gemm_split_z<V><<<split_blocks, 256, 0, s>>>(z_ref, c->n, zpad, recs, prec_terms(PREC),
                                                   static_cast<__nv_bfloat16*>(zp));
  RF_LAUNCHED();
  // one TMA box = a chunk's nH records of every (plane, term): dims (record bytes / EB, records,
  // planes x terms)
  const CUtensorMap zmap = gemm_tensor_map(zp, TF, recs, 2 * prec_terms(PREC), hankel_cores(PREC, KC));
  fn<<<grid, kGemmThreads, smem, s>>>(zmap, zpad, c->n, kern->gemm_B.as<unsigned char>(), KC, NCK, LP, kern->k,
                                      kern->lag0_d.as<int>(), TM, z_out, keys, W, nw, cols, c->status.as<int>());
  RF_LAUNCHED();
}

// Layouts: 16-neighbour groups with the widest output-shift stack, or the widest groups
// without shifts.
template <typename V, int PREC, bool WINMAX>
void launch_gemm_nj(rf_ctx* c, const rf_kernels* kern, const V* z_ref, V* z_out, unsigned long long* keys, int64_t W,
                    int64_t nw, cudaStream_t s) {
  constexpr int NJMAX = gemm_nj_max(PREC);
  constexpr int SMAX = gemm_shifts_max(PREC, 16);
  if (kern->gemm_NJ == 16) {
    RF_REQUIRE(kern->gemm_S == SMAX, "tensor-core form: unexpected shift count %d", kern->gemm_S);
    launch_gemm<V, 16, PREC, WINMAX, SMAX>(c, kern, z_ref, z_out, keys, W, nw, s);
  } else {
    RF_REQUIRE(kern->gemm_S == 1 && kern->gemm_NJ == NJMAX, "tensor-core form: unexpected layout");
    launch_gemm<V, NJMAX, PREC, WINMAX, 1>(c, kern, z_ref, z_out, keys, W, nw, s);
  }
}

template <typename V, bool WINMAX>
void launch_gemm_prec(rf_ctx* c, const rf_kernels* kern, int prec, const V* z_ref, V* z_out,
                      unsigned long long* keys, int64_t W, int64_t nw, cudaStream_t s) {
  switch (prec) {
    case RF_PREC_BF16: launch_gemm_nj<V, RF_PREC_BF16, WINMAX>(c, kern, z_ref, z_out, keys, W, nw, s); break;
    case RF_PREC_BF16X3: launch_gemm_nj<V, RF_PREC_BF16X3, WINMAX>(c, kern, z_ref, z_out, keys, W, nw, s); break;
    case RF_PREC_BF16X6: launch_gemm_nj<V, RF_PREC_BF16X6, WINMAX>(c, kern, z_ref, z_out, keys, W, nw, s); break;
    case RF_PREC_3XTF32: launch_gemm_nj<V, RF_PREC_3XTF32, WINMAX>(c, kern, z_ref, z_out, keys, W, nw, s); break;
    default: launch_gemm_nj<V, RF_PREC_BF16X9, WINMAX>(c, kern, z_ref, z_out, keys, W, nw, s); break;
  }
}

// Health check of the timeout path: waits, with a short limit, on an mbarrier that nothing
// arrives on, and records RF_ETIMEOUT in the status word exactly as a timed-out wait of the
// tensor-core kernel does.  Holds no tensor memory and issues no asynchronous copies.
__global__ void k_wait_selftest(int limit, int* __restrict__ status) {
  __shared__ __align__(8) unsigned long long mbar;
  const uint32_t addr = smem_u32(&mbar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(addr));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool done = mbar_wait(addr, 0u, limit);
  if (!__syncthreads_and(done) && threadIdx.x == 0) atomicExch(status, (int)RF_ETIMEOUT);
}

}  // namespace

void wait_selftest(rf_ctx* c, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(1024, c->status.as<int>());
  RF_LAUNCHED();
}

size_t gemm_zplanes_bytes(int64_t n, int64_t LP, int prec) {
  return (size_t)128 * (size_t)(2 * prec_terms(prec)) * (size_t)gemm_zrecs(n, LP, prec_tf32(prec)) + 256;
}

int gemm_max_len() { return 1 << 16; }

// The two tile layouts of a precision: (16 neighbours, the widest output-shift stack) and (the
// widest group, no shifts); (0, 0) leaves the choice to the rule of gemm_prepare.
bool gemm_layout_ok(int prec, int nj, int s) {
  if (nj == 0 && s == 0) return true;
  int smax = 1;
  switch (prec) {
    case RF_PREC_BF16: smax = gemm_shifts_max(RF_PREC_BF16, 16); break;
    case RF_PREC_BF16X3: smax = gemm_shifts_max(RF_PREC_BF16X3, 16); break;
    case RF_PREC_BF16X6: smax = gemm_shifts_max(RF_PREC_BF16X6, 16); break;
    case RF_PREC_3XTF32: smax = gemm_shifts_max(RF_PREC_3XTF32, 16); break;
    default: smax = gemm_shifts_max(RF_PREC_BF16X9, 16); break;
  }
  return (nj == 16 && s == smax && smax > 1) || (nj == gemm_nj_max(prec) && s == 1);
}

int gemm_stacked_shifts(int prec) {
  switch (prec) {
    case RF_PREC_BF16: return gemm_shifts_max(RF_PREC_BF16, 16);
    case RF_PREC_BF16X3: return gemm_shifts_max(RF_PREC_BF16X3, 16);
    case RF_PREC_BF16X6: return gemm_shifts_max(RF_PREC_BF16X6, 16);
    case RF_PREC_3XTF32: return gemm_shifts_max(RF_PREC_3XTF32, 16);
    default: return gemm_shifts_max(RF_PREC_BF16X9, 16);
  }
}

int gemm_wide_nj(int prec) { return gemm_nj_max(prec); }

void gemm_prepare(rf_ctx* c, rf_kernels* kern, int prec, cudaStream_t s) {
  const int terms = prec_terms(prec);
  const bool tf32 = prec_tf32(prec);
  // Layout: up to 16 neighbours with kernels longer than one 128-output tile take 16-wide
  // groups with the widest output-shift stack S (MMAs per output scale as
  // (LP + 128 (S - 1)) / S); otherwise the widest groups and no shifts.  K chunks of up to 128
  // taps (a power of two, so that they divide the 128 (S - 1) extension), halved while the
  // block's shared memory would keep a second block (as many as tensor memory admits) off
  // the SM.
  const int L16 = std::max(16, (kern->max_len + 15) / 16 * 16);
  int KC = 16;
  while (KC < 128 && KC < L16) KC *= 2;
  // a requested layout (the autotuner times both) replaces the rule
  const bool stack = kern->gemm_pref_nj ? kern->gemm_pref_nj == 16 && kern->gemm_pref_s > 1
                                        : kern->k <= 16 && L16 > kGemmM;
  const int NJ = stack ? 16 : gemm_nj_max(prec);
  int S = 1;
  if (stack) {
    switch (prec) {
      case RF_PREC_BF16: S = gemm_shifts_max(RF_PREC_BF16, 16); break;
      case RF_PREC_BF16X3: S = gemm_shifts_max(RF_PREC_BF16X3, 16); break;
      case RF_PREC_BF16X6: S = gemm_shifts_max(RF_PREC_BF16X6, 16); break;
      case RF_PREC_3XTF32: S = gemm_shifts_max(RF_PREC_3XTF32, 16); break;
      default: S = gemm_shifts_max(RF_PREC_BF16X9, 16); break;
    }
  }
  const size_t smem_cap = (size_t)(gemm_tmem_cols(prec, NJ, S) <= 256 ? 110 : 160) * 1024;
  while (KC > 16 && gemm_smem_bytes(prec, NJ, S, KC) > smem_cap) KC /= 2;
  const int LP = KC * ((L16 + KC - 1) / KC);
  const int NCK = (LP + kGemmM * (S - 1)) / KC;
  RF_REQUIRE(gemm_smem_bytes(prec, NJ, S, KC) <= 220 * 1024,
             "tensor-core direct form: chunk of %d taps does not fit", KC);
  if (kern->gemm_ready && kern->gemm_terms == terms && kern->gemm_tf32 == tf32 && kern->gemm_KC == KC &&
      kern->gemm_NCK == NCK && kern->gemm_NJ == NJ && kern->gemm_S == S && kern->gemm_LP == LP) {
    kern->gemm_prec = prec;  // same operands (the split terms serve every precision of the count)
    return;
  }
  const int groups = std::max(1, (kern->k + NJ - 1) / NJ);
  const int NC = S * 2 * NJ;
  const size_t elems = (size_t)groups * 2 * terms * NC * ((size_t)KC * NCK);
  kern->gemm_B.ensure((size_t)prec_ebytes(prec) * std::max<size_t>(elems, 8));
  dim3 grid((unsigned)std::max<int64_t>(1, ((int64_t)NC * KC * NCK + 255) / 256), (unsigned)groups);
  if (kern->dtype == RF_F64)
    k_gemm_prep_b<double2><<<grid, 256, 0, s>>>(kern->taps.p, kern->real, kern->off_d.as<int64_t>(),
                                                kern->len_d.as<int>(), kern->k, NJ, S, KC, NCK, LP, terms, tf32,
                                                kern->gemm_B.as<unsigned char>());
  else
    k_gemm_prep_b<float2><<<grid, 256, 0, s>>>(kern->taps.p, kern->real, kern->off_d.as<int64_t>(),
                                               kern->len_d.as<int>(), kern->k, NJ, S, KC, NCK, LP, terms, tf32,
                                               kern->gemm_B.as<unsigned char>());
  RF_LAUNCHED();
  RF_CUDA(cudaStreamSynchronize(s));
  kern->gemm_ready = true;
  kern->gemm_prec = prec;
  kern->gemm_terms = terms;
  kern->gemm_tf32 = tf32;
  kern->gemm_KC = KC;
  kern->gemm_NCK = NCK;
  kern->gemm_NJ = NJ;
  kern->gemm_S = S;
  kern->gemm_LP = LP;
}

void reconstruct_gemm(rf_ctx* c, const void* z_ref, rf_kernels* kern, int prec, void* z_out, int64_t W,
                      float* max_out, int32_t* argmax_out, cudaStream_t s) {
  if (kern->k == 0) return;
  RF_REQUIRE(c->n % kGemmM == 0, "the tensor-core direct form needs n to be a multiple of 128");
  gemm_prepare(c, kern, prec, s);  // no-op when the kernel set is prepared for this precision
  const bool win = max_out != nullptr;
  const int64_t nw = win ? (c->n + W - 1) / W : 0;
  unsigned long long* keys = nullptr;
  if (win) {
    c->scratch.ensure(sizeof(unsigned long long) * (size_t)kern->k * nw + 256);
    keys = c->scratch.as<unsigned long long>();
    RF_CUDA(cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * (size_t)kern->k * nw, s));
  }
  auto go = [&](auto vtag) {
    using V = decltype(vtag);
    const V* zr = static_cast<const V*>(z_ref);
    V* zo = static_cast<V*>(z_out);
    if (win) launch_gemm_prec<V, true>(c, kern, prec, zr, nullptr, keys, W, nw, s);
    else launch_gemm_prec<V, false>(c, kern, prec, zr, zo, nullptr, 0, 0, s);
  };
  if (c->g.dtype == RF_F64) go(double2{});
  else go(float2{});
  if (win) {
    const int64_t count = (int64_t)kern->k * nw;
    k_gemm_unpack<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(keys, count, max_out, argmax_out);
    RF_LAUNCHED();
  }
}

}  // namespace rf
