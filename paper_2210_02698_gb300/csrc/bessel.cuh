// bessel.cuh - FP64 Hankel functions H0^(1), H1^(1) of a positive real
// argument, for the Hankel-type functions f0, f1 of the HB ansatz
// (Eq. termf: f0 = i sqrt(pi)/2 H0(w tau), f1 = -i sqrt(pi)/2 (2 tau/w) H1(w tau)).
//
// Written from the mathematics (Abramowitz & Stegun, ch. 9), not from any
// library's implementation:
//  * x < HB_BESSEL_SWITCH: J_n by Miller's backward recurrence
//    J_{n-1} = (2n/x) J_n - J_{n+1} from an even start order M(x) with the
//    normalisation J0 + 2 sum_k J_2k = 1 (A&S 9.1.27, 9.1.46); Y0 by
//    Neumann's series (A&S 9.1.88)
//        Y0 = (2/pi)(ln(x/2) + gamma) J0 - (4/pi) sum_{k>=1} (-1)^k J_2k / k,
//    and Y1 = -Y0' from it, using J0' = -J1 and 2 J_n' = J_{n-1} - J_{n+1}:
//        Y1 = (2/pi)[(ln(x/2) + gamma - 1) J1 - J0/x]
//             + (2/pi) sum_{k>=2} (-1)^k (2k-1)/(k(k-1)) J_{2k-1}.
//  * x >= HB_BESSEL_SWITCH: Hankel's asymptotic expansion (A&S 9.2.5-9.2.10)
//        H_nu = sqrt(2/(pi x)) (P + iQ) e^{i(x - nu pi/2 - pi/4)},
//        P = sum_k (-1)^k a_2k / x^2k,  Q = sum_k (-1)^k a_{2k+1} / x^{2k+1},
//        a_k = prod_{j=1..k} (4nu^2 - (2j-1)^2) / (k! 8^k),
//    summed until the term falls below 1e-17 (the least term near k = 2x is
//    about e^{-2x}, far below FP64 rounding for x >= 25).  The phase uses one
//    FP64 sincos of x (argument reduction by the math library) rotated by
//    -pi/4 and -3pi/4.
// Both branches are FP64 throughout; absolute error ~1e-15 on the tested
// range [1e-3, 3e3] (tests compare against scipy/mpmath).
#pragma once
#include <math.h>

#ifdef __CUDACC__
#define HB_HD __host__ __device__ __forceinline__
#else
#define HB_HD inline
#endif

namespace hb {

constexpr double HB_BESSEL_SWITCH = 25.0;
constexpr double HB_PI = 3.14159265358979323846;
constexpr double HB_EULER_GAMMA = 0.57721566490153286061;
constexpr double HB_SQRT1_2 = 0.70710678118654752440;

struct Bessel01 {
  double j0, y0, j1, y1;
};

HB_HD void hb_sincos(double x, double* s, double* c) {
#ifdef __CUDA_ARCH__
  sincos(x, s, c);
#else
  *s = sin(x);
  *c = cos(x);
#endif
}

// Miller + Neumann branch, 0 < x < HB_BESSEL_SWITCH.
HB_HD Bessel01 bessel01_miller(double x) {
  const int M = 2 * (int)(0.8 * x + 13.0);          // even start order >= 26
  const double two_over_x = 2.0 / x;
  double tp1 = 0.0, t = 1e-30;                       // t_{n+1}, t_n at n = M
  double norm = 0.0, sy0 = 0.0, sy1 = 0.0, t1 = 0.0;
  for (int n = M; n >= 1; --n) {
    if ((n & 1) == 0) {
      const int k = n >> 1;
      norm += 2.0 * t;
      sy0 += ((k & 1) ? -t : t) / (double)k;
    } else {
      const int k = (n + 1) >> 1;
      if (k >= 2) {
        const double c = (double)(2 * k - 1) / ((double)k * (double)(k - 1));
        sy1 += ((k & 1) ? -c : c) * t;
      } else {
        t1 = t;
      }
    }
    const double tm1 = (double)n * two_over_x * t - tp1;
    tp1 = t;
    t = tm1;
    if (fabs(t) > 1e250) {
      t *= 1e-250; tp1 *= 1e-250; norm *= 1e-250; sy0 *= 1e-250; sy1 *= 1e-250; t1 *= 1e-250;
    }
  }
  norm += t;                                          // + J0 (unnormalised)
  const double sc = 1.0 / norm;
  Bessel01 r;
  r.j0 = t * sc;
  r.j1 = t1 * sc;
  const double lg = log(0.5 * x) + HB_EULER_GAMMA;
  r.y0 = (2.0 / HB_PI) * (lg * r.j0 - 2.0 * sy0 * sc);
  r.y1 = (2.0 / HB_PI) * ((lg - 1.0) * r.j1 - r.j0 / x + sy1 * sc);
  return r;
}

// Hankel asymptotic branch, x >= HB_BESSEL_SWITCH.
HB_HD Bessel01 bessel01_asym(double x) {
  const double inv8x = 0.125 / x;
  double b0 = 1.0, b1 = 1.0;                          // running a_k(nu) / x^k
  double P0 = 1.0, Q0 = 0.0, P1 = 1.0, Q1 = 0.0;
  for (int k = 1; k < 60; ++k) {
    const double odd = (double)(2 * k - 1);
    const double f = inv8x / (double)k;
    b0 *= (0.0 - odd * odd) * f;
    b1 *= (4.0 - odd * odd) * f;
    // k even -> P with sign (-1)^(k/2); k odd -> Q with sign (-1)^((k-1)/2)
    const double sg = ((k >> 1) & 1) ? -1.0 : 1.0;
    if (k & 1) { Q0 += sg * b0; Q1 += sg * b1; }
    else       { P0 += sg * b0; P1 += sg * b1; }
    if (fabs(b0) < 1e-17 && fabs(b1) < 1e-17) break;
  }
  double s, c;
  hb_sincos(x, &s, &c);
  const double amp = sqrt(2.0 / (HB_PI * x));
  const double c0 = (c + s) * HB_SQRT1_2, s0 = (s - c) * HB_SQRT1_2;   // chi0 = x - pi/4
  const double c1 = (s - c) * HB_SQRT1_2, s1 = -(s + c) * HB_SQRT1_2;  // chi1 = x - 3pi/4
  Bessel01 r;
  r.j0 = amp * (P0 * c0 - Q0 * s0);
  r.y0 = amp * (P0 * s0 + Q0 * c0);
  r.j1 = amp * (P1 * c1 - Q1 * s1);
  r.y1 = amp * (P1 * s1 + Q1 * c1);
  return r;
}

HB_HD Bessel01 bessel01(double x) {
  return (x < HB_BESSEL_SWITCH) ? bessel01_miller(x) : bessel01_asym(x);
}

#ifdef __CUDACC__
// g = v0 f0 + v1 f1 from interpolated tau^2, v0, v1 (Eq. babich, Eq. termf).
__device__ __forceinline__ double2 hb_green(double t2, double v0, double v1, double omega) {
  const double tau = sqrt(fmax(t2, 0.0));
  const double x = fmax(omega * tau, 1e-12);
  const Bessel01 b = bessel01(x);
  const double c = 0.88622692545275801365;         // sqrt(pi)/2
  const double k1 = c * 2.0 * tau / omega;
  // f0 = c(-Y0 + i J0),  f1 = k1 (Y1 - i J1)
  return make_double2(-c * b.y0 * v0 + k1 * b.y1 * v1, c * b.j0 * v0 - k1 * b.j1 * v1);
}
#endif

}  // namespace hb
