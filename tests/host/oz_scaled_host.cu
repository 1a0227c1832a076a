// Host driver for the split epilogue's scaled-integer term (paper_2509_23018_gb300/csrc/
// oz_digits.cuh, oz_scaled_int): reads lines "<val> <ex>" and prints the IEEE bits of
// val 2^max(-1022, ex) as 16 hex digits.  Built and run by tests/test_digits.py on the CPU.
#include <cstdio>
#include "../../paper_2509_23018_gb300/csrc/oz_digits.cuh"

int main()
{
    int val, ex;
    while (std::scanf("%d %d", &val, &ex) == 2) std::printf("%016llx\n", gw::oz_dbits(gw::oz_scaled_int(val, ex)));
    return 0;
}
