// Host-only brute-force check of pic::fast_div (the division used by the kernels to split
// cell indices): every divisor 1..4096 against dividends 0..65535 and random 31-bit
// dividends, plus random divisors up to 2^31 - 1.  Exit status 0 when all agree.
#include <cstdio>
#include <cstdlib>

#include "../../paper_0909_5603_gb300/csrc/pic_internal.h"

static unsigned long long state = 0x243F6A8885A308D3ULL;
static unsigned next32()
{
    state = state * 6364136223846793005ULL + 1442695040888963407ULL;
    return (unsigned)(state >> 33);
}

static int check(int d)
{
    const pic::FastDiv f = pic::make_fastdiv(d);
    for (int x = 0; x < 65536; ++x)
        if (pic::fast_div(x, f) != x / d) return 1;
    for (int t = 0; t < 4096; ++t) {
        const int x = (int)(next32() & 0x7fffffffu);
        if (pic::fast_div(x, f) != x / d) return 1;
    }
    const int edge[] = {0x7fffffff, 0x7ffffffe, d - 1, d, 2 * (d & 0x3fffffff) - 1};
    for (int x : edge)
        if (x >= 0 && pic::fast_div(x, f) != x / d) return 1;
    return 0;
}

int main()
{
    for (int d = 1; d <= 4096; ++d)
        if (check(d)) {
            printf("mismatch for divisor %d\n", d);
            return 1;
        }
    for (int t = 0; t < 2000; ++t) {
        const int d = 1 + (int)(next32() % 0x7ffffffeu);
        if (check(d)) {
            printf("mismatch for divisor %d\n", d);
            return 1;
        }
    }
    printf("fast_div ok\n");
    return 0;
}
