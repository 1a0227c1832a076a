// Host driver for the split's digit step (paper_2509_23018_gb300/csrc/oz_digits.cuh): reads
// lines "<x as 16 hex digits of its IEEE bits> <column max bits> <s>" and prints, per line, the
// column exponent E and the s digits as BF16 bit patterns (d_0 first).  Built and run by
// tests/test_digits.py on the CPU.
#include <cstdio>
#include "../../paper_2509_23018_gb300/csrc/oz_digits.cuh"

int main()
{
    unsigned long long xb, cb;
    int s;
    while (std::scanf("%llx %llx %d", &xb, &cb, &s) == 3) {
        const double x = gw::oz_bits_d(xb), cmax = gw::oz_bits_d(cb);
        const int E = gw::oz_expo_pos(cmax, -400);
        uint16_t d[8];
        gw::oz_store_digits(gw::oz_round_scaled(x, 6 * s - E), s, gw::oz_digit_bias(s), d, 1);
        std::printf("%d", E);
        for (int i = 0; i < s; ++i) std::printf(" %04x", d[i]);
        std::printf("\n");
    }
    return 0;
}
