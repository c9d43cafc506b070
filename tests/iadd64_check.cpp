// Checks dirac::iadd_rn (binary64 addition on the integer units) against the host's hardware addition, bit for
// bit, on random operand pairs drawn to reach every path: all exponents, exponent differences 0-70, exact and
// ulp-level cancellation, sums near rounding ties, tiny and huge operands, and the special values.
// Usage: iadd64_check [pairs]; exit status 0 when every pair agrees.
#include "iadd64.cuh"
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <random>
using namespace dirac;
static uint64_t bad = 0, tot = 0;
static void cmp(double h, double s, double a, double b, const char *op) {
    ++tot;
    if (iadd_bits(h) != iadd_bits(s) && !(std::isnan(h) && std::isnan(s))) {
        if (bad < 10) printf("MISMATCH %s a=%a b=%a hw=%a int=%a\n", op, a, b, h, s);
        ++bad;
    }
}
static void chk(double a, double b) {
    volatile double va = a, vb = b;
    cmp(va + vb, iadd_rn(a, b), a, b, "add");
    cmp(va - vb, isub_rn(a, b), a, b, "sub");
}
int main(int argc, char **argv) {
    long n = argc > 1 ? atol(argv[1]) : 10000000;
    std::mt19937_64 g(12345);
    auto rnd_in = [&](int e_lo, int e_hi) {
        uint64_t m = g() & ((1ull << 52) - 1);
        int sh = g() % 4;
        if (sh == 1) m &= ~((1ull << (g() % 52)) - 1);  // trailing zeros
        if (sh == 2) m |= ((1ull << (g() % 52)) - 1);   // trailing ones
        uint64_t e = e_lo + g() % (e_hi - e_lo + 1);
        uint64_t s = g() & 1;
        return iadd_double((s << 63) | (e << 52) | m);
    };
    for (long i = 0; i < n; ++i) {
        int mode = i % 6;
        double a, b;
        if (mode == 0) { a = rnd_in(1, 2046); b = rnd_in(1, 2046); }
        else if (mode == 1) { int e = 900 + g() % 200; a = rnd_in(e, e); b = rnd_in(e - (int)(g() % 70), e); }
        else if (mode == 2) { int e = 900 + g() % 200; a = rnd_in(e, e); b = -a * (1 + (double)(g() % 8 - 4) * 0x1p-52); }
        else if (mode == 3) {  // near ties: b = an odd multiple of a's half, quarter or eighth ulp
            int e = 900 + g() % 200; a = rnd_in(e, e); int k = 53 + g() % 3; b = ldexp((double)((g() % 7) | 1), e - 1023 - k) * ((g() & 1) ? 1 : -1); }
        else if (mode == 4) { a = rnd_in(0, 80); b = rnd_in(0, 80); }
        else { a = rnd_in(2040, 2047); b = rnd_in(2040, 2047); }
        chk(a, b); chk(b, a);
    }
    // specials
    double sp[] = {0.0, -0.0, 1.0, -1.0, INFINITY, -INFINITY, NAN, 0x1p-1074, -0x1p-1074, 0x1p-1022, 0x1.fffffffffffffp1023, -0x1.fffffffffffffp1023, 0x1p-960, 0x1p-959, 3.0, 0x1.0000000000001p0};
    for (double x : sp) for (double y : sp) chk(x, y);
    printf("checked %lu pairs, %lu mismatches\n", (unsigned long)tot, (unsigned long)bad);
    return bad != 0;
}
