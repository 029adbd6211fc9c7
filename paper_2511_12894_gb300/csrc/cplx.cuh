// Complex helpers and in-register small DFTs (radix 2, 4, 8, 16) used by the
// FFT passes and the overlap-save block transforms.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>
#include <utility>

namespace rf {

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };

template <typename V> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };

template <typename V> __host__ __device__ __forceinline__ V cmake(typename real_of<V>::type x, typename real_of<V>::type y) {
  V r; r.x = x; r.y = y; return r;
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return cmake<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return cmake<V>(a.x - b.x, a.y - b.y); }

// FP32 complex add / subtract as one paired-FP32 instruction (sm_100 and later): the same
// IEEE round-to-nearest results as two scalar operations, in one issue slot.
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) {
  float2 r;
  asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
  float2 r;
  asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return cmake<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {
  return cmake<V>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename V> __device__ __forceinline__ V cconj(V a) { return cmake<V>(a.x, -a.y); }
// twiddle from a table of exp(-2 pi i m / N): the table value for SIGN = -1, its conjugate for +1
template <int SIGN, typename V> __device__ __forceinline__ V tw_apply(V a, V w) {
  if constexpr (SIGN < 0) return cmul(a, w);
  else return cmulc(a, w);
}

// ---------------------------------------------------------------- compile-time loops
template <int I, int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

// exp(SIGN * 2 pi i Q / 16) applied to a, Q in [0, 16).  Exact for the multiples
// of pi/2; the other angles use the correctly rounded constants of cos/sin(k pi / 8).
template <int Q, int SIGN, typename V>
__device__ __forceinline__ V rot16(V a) {
  using R = typename real_of<V>::type;
  constexpr int q = ((Q % 16) + 16) % 16;
  if constexpr (q == 0) {
    return a;
  } else if constexpr (q == 4) {
    return cmake<V>(-SIGN * a.y, SIGN * a.x);
  } else if constexpr (q == 8) {
    return cmake<V>(-a.x, -a.y);
  } else if constexpr (q == 12) {
    return cmake<V>(SIGN * a.y, -SIGN * a.x);
  } else {
    // cos(2 pi q / 16), sin(2 pi q / 16)
    constexpr double C1 = 0.92387953251128675613;  // cos(pi/8)
    constexpr double S1 = 0.38268343236508977173;  // sin(pi/8)
    constexpr double H = 0.70710678118654752440;   // cos(pi/4)
    constexpr double cs[16] = {1, C1, H, S1, 0, -S1, -H, -C1, -1, -C1, -H, -S1, 0, S1, H, C1};
    constexpr double sn[16] = {0, S1, H, C1, 1, C1, H, S1, 0, -S1, -H, -C1, -1, -C1, -H, -S1};
    const R c = (R)cs[q];
    const R s = (R)(SIGN * sn[q]);
    return cmake<V>(a.x * c - a.y * s, a.x * s + a.y * c);
  }
}

// In-place DFT of R values in registers, natural order in and out:
//   y[k] = sum_n a[n] exp(SIGN 2 pi i n k / R).
template <int R, int SIGN, typename V>
__device__ __forceinline__ void dft(V* a);

template <int SIGN, typename V>
__device__ __forceinline__ void dft2(V& a0, V& a1) {
  V t = a0;
  a0 = cadd(t, a1);
  a1 = csub(t, a1);
}

template <int SIGN, typename V>
__device__ __forceinline__ void dft4(V& a0, V& a1, V& a2, V& a3) {
  V t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3);
  V d = csub(a1, a3);
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  // t1 +- d * (SIGN i), written out so the quarter turn costs no moves
  a1 = cmake<V>(t1.x - SIGN * d.y, t1.y + SIGN * d.x);
  a3 = cmake<V>(t1.x + SIGN * d.y, t1.y - SIGN * d.x);
}

// R = R1 * R2 with n = n1 + R1 n2, k = k2 + R2 k1.
template <int R1, int R2, int SIGN, typename V>
__device__ __forceinline__ void dft_split(V* a) {
  constexpr int R = R1 * R2;
  V b[R];
  // inner DFTs of length R2 over n2 for each n1, then twiddle exp(SIGN 2 pi i n1 k2 / R)
  static_for<0, R1>([&](auto n1c) {
    constexpr int n1 = decltype(n1c)::value;
    V t[R2];
    static_for<0, R2>([&](auto n2c) { constexpr int n2 = decltype(n2c)::value; t[n2] = a[n1 + R1 * n2]; });
    if constexpr (R2 == 2) dft2<SIGN>(t[0], t[1]);
    else if constexpr (R2 == 4) dft4<SIGN>(t[0], t[1], t[2], t[3]);
    static_for<0, R2>([&](auto k2c) {
      constexpr int k2 = decltype(k2c)::value;
      b[n1 * R2 + k2] = rot16<(n1 * k2 * (16 / R)) % 16, SIGN>(t[k2]);
    });
  });
  // outer DFTs of length R1 over n1 for each k2
  static_for<0, R2>([&](auto k2c) {
    constexpr int k2 = decltype(k2c)::value;
    V t[R1];
    static_for<0, R1>([&](auto n1c) { constexpr int n1 = decltype(n1c)::value; t[n1] = b[n1 * R2 + k2]; });
    if constexpr (R1 == 2) dft2<SIGN>(t[0], t[1]);
    else if constexpr (R1 == 4) dft4<SIGN>(t[0], t[1], t[2], t[3]);
    static_for<0, R1>([&](auto k1c) { constexpr int k1 = decltype(k1c)::value; a[k2 + R2 * k1] = t[k1]; });
  });
}

template <int R, int SIGN, typename V>
__device__ __forceinline__ void dft(V* a) {
  static_assert(R == 2 || R == 4 || R == 8 || R == 16, "radix");
  if constexpr (R == 2) dft2<SIGN>(a[0], a[1]);
  else if constexpr (R == 4) dft4<SIGN>(a[0], a[1], a[2], a[3]);
  else if constexpr (R == 8) dft_split<2, 4, SIGN>(a);
  else dft_split<4, 4, SIGN>(a);
}

}  // namespace rf
