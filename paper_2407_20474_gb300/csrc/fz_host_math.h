// fz_host_math.h -- host-side integer helpers of the closed forms, with no
// CUDA dependency (the CPU tests compile this header on its own).
#pragma once

#include <cstdint>

namespace fz {

// Extended Euclid for the last two generators (g, h) >= 1: e = gcd(g, h),
// h1 = h / e, g1 = g / e and inv = g1^-1 mod h1 (0 when h1 = 1).  The
// a_{d-2} of Z(p, (g, h)) are the v = (p / e) inv (mod h1) up to p / g
// (when e divides p), the walk-leaf progression and the pair memo.
inline void pair_params(int64_t g, int64_t h, int64_t *e_out, int64_t *h1_out, int64_t *g1_out,
                        int64_t *inv_out) {
    // x g + y h = e
    int64_t r0 = g, r1 = h, x0 = 1, x1 = 0;
    while (r1 != 0) {
        const int64_t q = r0 / r1;
        int64_t t = r0 - q * r1;
        r0 = r1;
        r1 = t;
        t = x0 - q * x1;
        x0 = x1;
        x1 = t;
    }
    const int64_t e = r0, h1 = h / e;
    int64_t inv = h1 > 1 ? x0 % h1 : 0;
    if (inv < 0) inv += h1;
    *e_out = e;
    *h1_out = h1;
    *g1_out = g / e;
    *inv_out = inv;
}

// Sum over i = 0..cnt-1 of floor((a i + b) / m), a, b >= 0, m >= 1 (the
// Euclid-like reduction of floor sums: take out the whole parts of a / m and
// b / m, then count the lattice points under the line the other way round).
inline unsigned __int128 floor_sum(uint64_t cnt, uint64_t m, uint64_t a, uint64_t b) {
    unsigned __int128 ans = 0;
    for (;;) {
        if (a >= m) {
            ans += (unsigned __int128)cnt * (cnt - 1) / 2 * (a / m);
            a %= m;
        }
        if (b >= m) {
            ans += (unsigned __int128)cnt * (b / m);
            b %= m;
        }
        const unsigned __int128 y = (unsigned __int128)a * cnt + b;
        if (y < m) break;
        cnt = (uint64_t)(y / m);
        b = (uint64_t)(y % m);
        const uint64_t t = m;
        m = a;
        a = t;
    }
    return ans;
}

// Rows of the pair's run-order memo up to element n >= 0: the points
// (x, y) >= 0 with t0 x + t1 y <= n, i.e. the sum over p <= n of
// |Z(p, (t0, t1))| (saturated at 2^64 - 1).
inline uint64_t pair_rows_upto(int64_t n, int64_t t0, int64_t t1) {
    const uint64_t X = (uint64_t)(n / t0);
    // sum over x <= X of floor((n - t0 x) / t1) + 1; with x' = X - x the
    // numerator is (n mod t0) + t0 x'
    const unsigned __int128 s =
        floor_sum(X + 1, (uint64_t)t1, (uint64_t)t0, (uint64_t)(n % t0)) + X + 1;
    return s > (unsigned __int128)~0ull ? ~0ull : (uint64_t)s;
}

}  // namespace fz
