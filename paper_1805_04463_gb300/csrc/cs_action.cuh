// cs_action.cuh -- Benincasa-Dowker action arithmetic shared by the
// single-set and batched action kernels and the host path (Section "The
// Benincasa-Dowker Action"), in double-double FP64.
#pragma once

#include <cmath>

#include "cs_internal.cuh"

namespace cs {

constexpr int kMaxEps = 16;  // eps values per call
constexpr int kActThreads = 256;
constexpr int kActBlocks = 128;

struct EpsArgs {
    double v[kMaxEps];
    int64_t kend[kMaxEps];  // smeared-sum cutoffs (single-set kernels; set on the host)
    int n;
};

__host__ __device__ inline dd dd_div(dd a, dd b) {
    const double q1 = a.hi / b.hi;
    dd r = dd_sub(a, dd_mul_d(b, q1));
    const double q2 = r.hi / b.hi;
    r = dd_sub(r, dd_mul_d(b, q2));
    const double q3 = r.hi / b.hi;
    return dd_add(dd_quick_two_sum(q1, q2), dd_from(q3));
}

// One Newton step on the correctly rounded double root: x + (a - x^2) / (2x).
__host__ __device__ inline dd dd_sqrt(dd a) {
    if (a.hi <= 0.0) return dd_from(0.0);
    const double x = sqrt(a.hi);
    const dd r = dd_sub(a, dd_two_prod(x, x));
    return dd_quick_two_sum(x, r.hi / (2.0 * x));
}

// The integer in parentheses of the local action; in 2+1 eight times it
// (8N - 8n1 + 27n2 - 18n3) so that it stays an integer.
__host__ __device__ inline int64_t bracket_of(int dim, int64_t n, const int64_t* h4) {
    if (dim == 2) return n - 2 * h4[0] + 4 * h4[1] - 2 * h4[2];
    if (dim == 3) return 8 * n - 8 * h4[0] + 27 * h4[1] - 18 * h4[2];
    return n - h4[0] + 9 * h4[1] - 16 * h4[2] + 8 * h4[3];
}

// The 2+1 constant (pi/(3 sqrt 2))^(2/3) / Gamma(5/3) of Eqs. s3d_local and
// b3d_local, from the math library in double (a constant factor; its
// rounding is ~1e-16 relative).
__host__ __device__ inline double c3_const() {
    const double v = cbrt(3.14159265358979323846 / (3.0 * sqrt(2.0)));
    return v * v / tgamma(5.0 / 3.0);
}

__host__ __device__ inline bool is_local(double eps) { return eps <= 0.0 || eps == 1.0; }

// Local action: 2 * bracket (1+1), c3 * bracket / 8 (2+1) or
// 4/sqrt(6) * bracket (3+1).
__host__ __device__ inline dd local_action(int dim, int64_t bracket) {
    const dd b = dd_from_i64(bracket);
    if (dim == 2) return dd_mul_d(b, 2.0);
    if (dim == 3) return dd_mul_d(b, c3_const() * 0.125);
    return dd_mul(dd_div(dd_from(4.0), dd_sqrt(dd_from(6.0))), b);
}

// Smeared action from sum = sum_k N_k f(k, eps):
//   1+1: 2 eps [N - 2 eps sum];  2+1: c3 eps^(2/3) [N - eps sum];
//   3+1: 4 sqrt(eps/6) [N - eps sum].
__host__ __device__ inline dd smeared_action(int dim, int64_t n, double eps, dd sum) {
    const dd e = dd_from(eps);
    if (dim == 2) {
        const dd inner = dd_sub(dd_from_i64(n), dd_mul(dd_mul_d(e, 2.0), sum));
        return dd_mul(dd_mul_d(e, 2.0), inner);
    }
    const dd inner = dd_sub(dd_from_i64(n), dd_mul(e, sum));
    if (dim == 3) {
        const double r = cbrt(eps);
        return dd_mul_d(inner, c3_const() * (r * r));
    }
    const dd pref = dd_mul_d(dd_sqrt(dd_div(e, dd_from(6.0))), 4.0);
    return dd_mul(pref, inner);
}

// Terms k >= K of the smeared sum that can be dropped.  For k >= deg,
// f_d(k) = q^(k-deg) poly_d(k) with q = 1 - eps and
//   |poly_2| <= (1 + k eps)^2, |poly_3| <= 3.375 (1 + k eps)^2,
//   |poly_4| <= 9 (1 + k eps)^3,
// so |f_d(k)| <= B(k) = C (1 + k eps)^m q^(k-deg), which decreases for
// k >= m / eps.  With R >= the sum of the abundances (n(n-1)/2 bounds it for
// any histogram of n elements) the dropped tail is at most R B(K), and the
// sum enters S multiplied by at most 4 (4 eps^2, c3 eps^(5/3) or
// 4 sqrt(eps/6) eps).  K is the first k >= max(deg, m/eps) with
// 4 R B(K) <= 1e-15: the truncation moves S by less than 1e-15.
__host__ __device__ inline int64_t smear_cutoff(int dim, double eps, double R, int64_t len) {
    const double lq = log1p(-eps);  // ln q < 0
    if (!(lq < 0.0)) return len;
    const double C = dim == 2 ? 1.0 : (dim == 3 ? 3.375 : 9.0);
    const double m = dim == 4 ? 3.0 : 2.0;
    const double deg = dim == 4 ? 3.0 : 2.0;
    const double lhs0 = log(4.0 * fmax(R, 1.0) * C) + 34.6;  // ln(4 R C) - ln(1e-15)
    double k = fmax(deg, ceil(m / eps));
    // Fixed point of k = deg + (lhs0 + m ln(1 + k eps)) / (-ln q), approached
    // from below; the map's slope there is about m / (1 + k eps) < 0.1.  The
    // iterates never decrease, and once one repeats every later one does, so
    // stopping there gives the same k as all 24 steps.
    for (int it = 0; it < 24; ++it) {
        const double kn = fmax(k, deg + (lhs0 + m * log1p(k * eps)) / -lq);
        if (kn == k) break;
        k = kn;
    }
    k = ceil(k) + 8.0;
    return k < double(len) ? int64_t(k) : len;
}


}  // namespace cs
