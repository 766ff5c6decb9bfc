// Host check of the fused transform's FastDiv (fastdiv.cuh) against integer
// division: every divisor 1..4096 (coefficient extents), all dividends below
// 2^16, dividends next to multiples of the divisor up to 2^24 (row indices
// N1 N2), and random 32-bit dividends.  Exit status 1 on any mismatch.
#include <cstdio>
#include <random>

#include "fastdiv.cuh"

int main() {
    std::mt19937_64 g(7);
    long long checked = 0, bad = 0;
    for (unsigned d = 1; d <= 4096; ++d) {
        const gbnfft::FastDiv f = gbnfft::make_fastdiv(d);
        auto check = [&](unsigned x) {
            ++checked;
            if (f.div(x) != x / d) {
                if (bad < 5) std::printf("mismatch d=%u x=%u: %u vs %u\n", d, x, f.div(x), x / d);
                ++bad;
            }
        };
        for (unsigned x = 0; x < (1u << 16); ++x) check(x);
        for (unsigned q = 1; q < (1u << 24) / d; q += 1 + q / 64) {
            const unsigned x = q * d;
            check(x - 1);
            check(x);
            check(x + 1);
        }
        for (int k = 0; k < 2000; ++k) check((unsigned)g());
        check(0xFFFFFFFFu);
    }
    std::printf("checked %lld mismatches %lld\n", checked, bad);
    return bad != 0;
}
