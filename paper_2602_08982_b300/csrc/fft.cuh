// Register-resident mixed-radix (2/3/4/5) DFTs for the spectral derivatives of
// Eq. derivative-spectral, and the cross-lane radix-2 stages that split one
// pencil of length N = N1 * T over T adjacent lanes (warp shuffles).
//
// Index conventions (forward transform, W_N = exp(-2 pi i / N)):
//   lane j of a pencil group holds x[j + T m], m = 0..N1-1.
//   After pencil_fwd, register k1 of lane j holds X[k1 + N1 * brev_T(j)].
//   pencil_inv consumes exactly that layout and returns x[j + T m] scaled by N
//   (unnormalised inverse); the caller folds 1/N into its multiplier.
#pragma once
#include <cuda_runtime.h>
#include <type_traits>

namespace wslda {

template <typename R> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename R> using cx = typename cplx_of<R>::type;

template <typename C> __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) { C r; r.x = a; r.y = b; return r; }
template <typename C> __device__ __forceinline__ C add(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C sub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C neg(C a) { return mk<C>(-a.x, -a.y); }
template <typename C> __device__ __forceinline__ C mul(C a, C b) { return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename C> __device__ __forceinline__ C mulc(C a, C b) { return mk<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }  // a * conj(b)
template <typename C> __device__ __forceinline__ C scl(C a, decltype(C::x) s) { return mk<C>(a.x * s, a.y * s); }
template <typename C> __device__ __forceinline__ C mul_mi(C a) { return mk<C>(a.y, -a.x); }   // a * (-i)
template <typename C> __device__ __forceinline__ C mul_pi(C a) { return mk<C>(-a.y, a.x); }   // a * (+i)

// ---------------------------------------------------------------------------
// Compile-time twiddles: cos(2 pi a / d) and sin(2 pi a / d) in double.
// The angle is reduced exactly (integer arithmetic) to [0, pi/4], then the
// Taylor series of cos or sin is summed; |x| <= pi/4 makes 14 terms far more
// than enough for double precision.
// ---------------------------------------------------------------------------
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double taylor_cos(double x) {
  double t = 1.0, s = 1.0;
  for (int k = 1; k < 14; ++k) { t *= -x * x / ((2.0 * k - 1.0) * (2.0 * k)); s += t; }
  return s;
}
constexpr double taylor_sin(double x) {
  double t = x, s = x;
  for (int k = 1; k < 14; ++k) { t *= -x * x / ((2.0 * k) * (2.0 * k + 1.0)); s += t; }
  return s;
}
constexpr double cos2pi(long long a, long long d) {
  long long D = 8 * d;
  long long A = (((a % d) + d) % d) * 8;
  if (2 * A > D) A = D - A;              // cos(2pi - x) = cos x
  double sg = 1.0;
  if (4 * A > D) { sg = -1.0; A = D / 2 - A; }   // cos(pi - x) = -cos x
  if (8 * A > D) return sg * taylor_sin(kTwoPi * double(D / 4 - A) / double(D));
  return sg * taylor_cos(kTwoPi * double(A) / double(D));
}
constexpr double sin2pi(long long a, long long d) { return cos2pi(4 * a - d, 4 * d); }

template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// a * W_N^E with W_N = exp(-2 pi i/N) (forward) or its conjugate (INV).
template <int N, int E, bool INV, typename C>
__device__ __forceinline__ C twiddle(C a) {
  constexpr int e = ((E % N) + N) % N;
  using R = decltype(C::x);
  if constexpr (e == 0) {
    return a;
  } else if constexpr (2 * e == N) {
    return neg(a);
  } else if constexpr (4 * e == N) {
    return INV ? mul_pi(a) : mul_mi(a);
  } else if constexpr (4 * e == 3 * N) {
    return INV ? mul_mi(a) : mul_pi(a);
  } else {
    constexpr double c = cos2pi(e, N);
    constexpr double s = INV ? sin2pi(e, N) : -sin2pi(e, N);
    return mk<C>(a.x * R(c) - a.y * R(s), a.x * R(s) + a.y * R(c));
  }
}

// P-point DFT in place, P in {2, 3, 4} with hand-written butterflies, other
// small primes by the direct sum with compile-time twiddles.
template <int P, bool INV, typename C>
__device__ __forceinline__ void butterfly(C* x) {
  using R = decltype(C::x);
  if constexpr (P == 2) {
    C a = x[0], b = x[1];
    x[0] = add(a, b);
    x[1] = sub(a, b);
  } else if constexpr (P == 3) {
    constexpr double h = 0.86602540378443864676372317075294;  // sin(2pi/3)
    C t1 = add(x[1], x[2]);
    C t2 = sub(x[0], scl(t1, R(0.5)));
    C d = scl(sub(x[1], x[2]), R(h));
    x[0] = add(x[0], t1);
    if constexpr (!INV) { x[1] = add(t2, mul_mi(d)); x[2] = add(t2, mul_pi(d)); }
    else { x[1] = add(t2, mul_pi(d)); x[2] = add(t2, mul_mi(d)); }
  } else if constexpr (P == 4) {
    C a = add(x[0], x[2]), b = sub(x[0], x[2]);
    C c = add(x[1], x[3]), d = sub(x[1], x[3]);
    x[0] = add(a, c);
    x[2] = sub(a, c);
    if constexpr (!INV) { x[1] = add(b, mul_mi(d)); x[3] = add(b, mul_pi(d)); }
    else { x[1] = add(b, mul_pi(d)); x[3] = add(b, mul_mi(d)); }
  } else {
    C y[P];
    static_for<0, P>([&](auto s) {
      constexpr int S = decltype(s)::value;
      C acc = x[0];
      static_for<1, P>([&](auto r) {
        constexpr int Rr = decltype(r)::value;
        acc = add(acc, twiddle<P, Rr * S, INV>(x[Rr]));
      });
      y[S] = acc;
    });
    static_for<0, P>([&](auto s) { x[decltype(s)::value] = y[decltype(s)::value]; });
  }
}

template <int N>
constexpr int first_radix() {
  return (N % 4 == 0 && N != 8) ? 4 : (N % 2 == 0) ? 2 : (N % 3 == 0) ? 3 : N;
}

// Unnormalised N-point DFT of a register array, natural order in and out
// (decimation in time: N = P * Q, Q-point DFTs of the P interleaved
// subsequences, twiddles W_N^{r k}, then P-point butterflies).
template <int N, bool INV, typename C>
__device__ __forceinline__ void dft(C* x) {
  if constexpr (N == 1) {
    return;
  } else if constexpr (N == 2 || N == 3 || N == 4 || N == 5) {
    butterfly<N, INV>(x);
  } else {
    constexpr int P = first_radix<N>();
    constexpr int Q = N / P;
    static_assert(P * Q == N && Q > 1, "radix-2/3/5 lengths only");
    C y[P][Q];
    static_for<0, P>([&](auto r) {
      constexpr int Rr = decltype(r)::value;
      static_for<0, Q>([&](auto m) { y[Rr][decltype(m)::value] = x[P * decltype(m)::value + Rr]; });
      dft<Q, INV>(y[Rr]);
    });
    static_for<0, Q>([&](auto k) {
      constexpr int K = decltype(k)::value;
      C t[P];
      static_for<0, P>([&](auto r) {
        constexpr int Rr = decltype(r)::value;
        t[Rr] = twiddle<N, Rr * K, INV>(y[Rr][K]);
      });
      butterfly<P, INV>(t);
      static_for<0, P>([&](auto s) { x[K + Q * decltype(s)::value] = t[decltype(s)::value]; });
    });
  }
}

__host__ __device__ constexpr int brev(int j, int T) {
  int r = 0;
  for (int b = 1; b < T; b <<= 1) { r <<= 1; if (j & b) r |= 1; }
  return r;
}

// Forward transform of one pencil split over T lanes (see header comment).
// tw[k] = W_N^k, k < N, only read when T > 1.
template <int N, int T, typename C>
__device__ __forceinline__ void pencil_fwd(C* x, int j, const C* tw) {
  constexpr int N1 = N / T;
  dft<N1, false>(x);
  if constexpr (T > 1) {
    static_for<1, N1>([&](auto k) {
      constexpr int K = decltype(k)::value;
      x[K] = mul(x[K], tw[(j * K) % N]);
    });
    static_for<0, 8>([&](auto st) {
      constexpr int h = (T >> 1) >> decltype(st)::value;
      if constexpr (h >= 1) {
        const bool upper = (j & h) != 0;
        const C w = tw[(j & (h - 1)) * (N / (2 * h))];
#pragma unroll
        for (int k = 0; k < N1; ++k) {
          C o;
          o.x = __shfl_xor_sync(0xffffffffu, x[k].x, h);
          o.y = __shfl_xor_sync(0xffffffffu, x[k].y, h);
          x[k] = upper ? mul(sub(o, x[k]), w) : add(x[k], o);
        }
      }
    });
  }
}

// Inverse of pencil_fwd up to the factor N.
template <int N, int T, typename C>
__device__ __forceinline__ void pencil_inv(C* x, int j, const C* tw) {
  constexpr int N1 = N / T;
  if constexpr (T > 1) {
    static_for<0, 8>([&](auto st) {
      constexpr int h = 1 << decltype(st)::value;
      if constexpr (h < T) {
        const bool upper = (j & h) != 0;
        const C w = tw[(j & (h - 1)) * (N / (2 * h))];
#pragma unroll
        for (int k = 0; k < N1; ++k) {
          C o;
          o.x = __shfl_xor_sync(0xffffffffu, x[k].x, h);
          o.y = __shfl_xor_sync(0xffffffffu, x[k].y, h);
          x[k] = upper ? sub(o, mulc(x[k], w)) : add(x[k], mulc(o, w));
        }
      }
    });
    static_for<1, N1>([&](auto k) {
      constexpr int K = decltype(k)::value;
      x[K] = mulc(x[K], tw[(j * K) % N]);
    });
  }
  dft<N1, true>(x);
}

}  // namespace wslda
