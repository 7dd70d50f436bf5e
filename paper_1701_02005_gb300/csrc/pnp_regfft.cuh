// Register FFTs (FP32 for the mixed path, FP64 for the FP64 path).
//
// A length-N transform is split N = R1 x G (Cooley-Tukey, one level): with
// n = g + G r and k = k1 + R1 k2,
//     X[k1 + R1 k2] = sum_g W_G^{g k2} ( W_N^{g k1} sum_r x[g + G r] W_R1^{r k1} ),
// W_M = exp(-2 pi i / M) (the inverse transform conjugates every W).  Each of
// G threads does an R1-point DFT of its strided samples in registers and
// multiplies by the twiddle W_N^{g k1}; after one exchange through shared
// memory the G-point DFTs over g run in registers again.  One shared-memory
// round trip per transform instead of one per radix-4 stage.
//
// The small DFTs are radix-2 decimation in frequency, unrolled by template
// recursion so that every twiddle is a compile-time constant; the constants
// come from a Taylor series of sin and cos on [0, pi/4] (octant symmetry),
// written here from the series itself and evaluated by the compiler.
#pragma once

#include <type_traits>

#include "pnp_common.cuh"

namespace pnp {
namespace rfft {

constexpr double kPi = 3.141592653589793238462643383279502884;

constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int n = 1; n < 16; ++n) {
    term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
    sum += term;
  }
  return sum;
}

constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int n = 1; n < 16; ++n) {
    term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
    sum += term;
  }
  return sum;
}

// cos a and sin a for a in [0, pi]
constexpr double cos_0pi(double a) {
  return a <= kPi / 4 ? taylor_cos(a)
         : a <= kPi / 2 ? taylor_sin(kPi / 2 - a)
         : a <= 3 * kPi / 4 ? -taylor_sin(a - kPi / 2)
                            : -taylor_cos(kPi - a);
}
constexpr double sin_0pi(double a) {
  return a <= kPi / 4 ? taylor_sin(a)
         : a <= kPi / 2 ? taylor_cos(kPi / 2 - a)
         : a <= 3 * kPi / 4 ? taylor_cos(a - kPi / 2)
                            : taylor_sin(kPi - a);
}

// cos and sin of 2 pi k / M; multiples of pi/2 exact
constexpr double cos2pi(int k, int M) {
  k %= M;
  if (k < 0) k += M;
  if ((4 * k) % M == 0) {
    const int q = 4 * k / M;
    return q == 0 ? 1.0 : q == 2 ? -1.0 : 0.0;
  }
  if (2 * k > M) k = M - k;   // cos(2 pi - a) = cos a
  return cos_0pi(2.0 * kPi * k / M);
}
constexpr double sin2pi(int k, int M) {
  k %= M;
  if (k < 0) k += M;
  if ((4 * k) % M == 0) {
    const int q = 4 * k / M;
    return q == 1 ? 1.0 : q == 3 ? -1.0 : 0.0;
  }
  if (2 * k > M) return -sin_0pi(2.0 * kPi * (M - k) / M);   // sin(2 pi - a) = -sin a
  return sin_0pi(2.0 * kPi * k / M);
}

constexpr int bitrev(int k, int M) {
  int r = 0;
  for (int m = M >> 1; m >= 1; m >>= 1) {
    r = (r << 1) | (k & 1);
    k >>= 1;
  }
  return r;
}

// z W_M^I (forward) or z conj(W_M^I) (inverse), W_M = exp(-2 pi i / M), in
// the precision T of the transform (float or double)
template <bool INV, int I, int M, typename T>
__host__ __device__ __forceinline__ cplx<T> twiddle(cplx<T> z) {
  if constexpr (I == 0) {
    return z;
  } else if constexpr (4 * I == M) {
    return INV ? cplx<T>{-z.y, z.x} : cplx<T>{z.y, -z.x};
  } else {
    constexpr T c = (T)cos2pi(I, M);
    constexpr T s = (INV ? T(1) : T(-1)) * (T)sin2pi(I, M);
    return {z.x * c - z.y * s, z.x * s + z.y * c};
  }
}

template <bool INV, int HALF, int B, int I, typename T>
__host__ __device__ __forceinline__ void dif_butterflies(cplx<T>* v) {
  if constexpr (I < HALF) {
    const cplx<T> a = v[B + I], c = v[B + I + HALF];
    v[B + I] = cadd(a, c);
    v[B + I + HALF] = twiddle<INV, I, 2 * HALF>(csub(a, c));
    dif_butterflies<INV, HALF, B, I + 1>(v);
  }
}

template <bool INV, int M, int HALF, int B, typename T>
__host__ __device__ __forceinline__ void dif_blocks(cplx<T>* v) {
  if constexpr (B < M) {
    dif_butterflies<INV, HALF, B, 0>(v);
    dif_blocks<INV, M, HALF, B + 2 * HALF>(v);
  }
}

template <bool INV, int M, int HALF, typename T>
__host__ __device__ __forceinline__ void dif_stages(cplx<T>* v) {
  if constexpr (HALF >= 1) {
    dif_blocks<INV, M, HALF, 0>(v);
    dif_stages<INV, M, HALF / 2>(v);
  }
}

// In-place M-point DFT of v[0..M); the result X[k] is left at v[bitrev(k, M)].
template <bool INV, int M, typename T>
__host__ __device__ __forceinline__ void dft(cplx<T>* v) {
  dif_stages<INV, M, M / 2>(v);
}

// f(std::integral_constant<int, I>) for I = B .. E-1: a loop whose index is a
// constant expression in the body
template <int B, int E, typename F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

}  // namespace rfft
}  // namespace pnp
