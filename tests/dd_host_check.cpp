// Host harness for the double-double arithmetic of the library (dd.cuh),
// compiled by tests/test_dd_host.py with the host compiler.  Reads lines
// "op a_hi a_lo b_hi b_lo" (hex floats) from stdin and prints the result
// pair "hi lo" in hex floats, for exact checking in rational arithmetic.
//   op = S: two_sum(a_hi, b_hi)   P: two_prod(a_hi, b_hi)
//        A: (a_hi + a_lo) + (b_hi + b_lo)   M: (a_hi + a_lo) * (b_hi + b_lo)
#define __host__
#define __device__
#define __forceinline__ inline
#include <cstdio>
#include <cstdlib>

#include "../paper_1607_03777_gb300/csrc/dd.cuh"

int main() {
    char op;
    char s1[64], s2[64], s3[64], s4[64];
    while (std::scanf(" %c %63s %63s %63s %63s", &op, s1, s2, s3, s4) == 5) {
        const double ah = std::strtod(s1, nullptr), al = std::strtod(s2, nullptr);
        const double bh = std::strtod(s3, nullptr), bl = std::strtod(s4, nullptr);
        double hi = 0.0, lo = 0.0;
        if (op == 'S') {
            sip::two_sum(ah, bh, hi, lo);
        } else if (op == 'P') {
            sip::two_prod(ah, bh, hi, lo);
        } else if (op == 'A' || op == 'M') {
            const sip::dd a(ah, al), b(bh, bl);
            const sip::dd c = op == 'A' ? a + b : a * b;
            hi = c.hi;
            lo = c.lo;
        } else {
            return 2;
        }
        std::printf("%a %a\n", hi, lo);
    }
    return 0;
}
