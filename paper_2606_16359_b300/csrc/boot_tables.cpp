// Twiddles of the bootstrapping's special-FFT stages as correctly rounded
// doubles: cos(pi e / N) evaluated in quad precision (113-bit significand) and
// rounded once to the nearest double.  Compiled as plain host C++ (quad
// precision via libquadmath).
#include <quadmath.h>

double boot_cos_pi_table_entry(int N, int e) {
    if (2 * e == N) return 0.0;  // cos(pi / 2) exactly
    const __float128 pi = 4 * atanq((__float128)1);
    return (double)cosq(pi * (__float128)e / (__float128)N);
}
