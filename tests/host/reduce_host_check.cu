// Host check of set_points' fixed-point coordinate reduction (reduce.cuh):
// for n = 2^L the integer path must give the same stencil origin and the
// same offset bits as the FP64 round-to-nearest steps
//     x_w = x - floor(x + 1/2), t = x_w + 1/2, u = n t, v = u - (m + 1/2),
//     l0 = ceil(v), s = l0 - v,
// on random, boundary and tie-producing inputs.  Prints the counts; exit
// status 1 on any mismatch.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>

#include "reduce.cuh"

using namespace gbnfft;

int main(int argc, char **argv) {
    const long long per = argc > 1 ? std::atoll(argv[1]) : 1000000;
    std::mt19937_64 g(2024);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    long long total = 0, fixed = 0, bad = 0;
    const int Ls[] = {3, 4, 5, 8, 9, 10, 12, 20, 30};
    const int ms[] = {1, 3, 6, 8};
    for (int L : Ls)
        for (int m : ms) {
            const CoordParams c = coord_params(1 << L, m);
            const double nd = c.nd, alpha = c.alpha;
            for (long long it = 0; it < per; ++it) {
                double x;
                switch (it % 6) {
                    case 0: x = U(g) - 0.5; break;
                    case 1: x = -0.5 + U(g) * std::ldexp(1.0, -8); break;   // t around 2^-10
                    case 2: {                                                // every exponent
                        const int e = -(int)(g() % 62) - 1;
                        x = std::ldexp(1.0 + U(g), e) * ((g() & 1) ? -1.0 : 1.0);
                        break;
                    }
                    case 3: {   // grid nodes, half nodes, u - alpha integral, and FP64 neighbours
                        const double l = (double)(g() % (unsigned long long)(nd + 5)) - 2.0;
                        const double off[3] = {0.0, 0.5, alpha};
                        x = (l + off[g() % 3]) / nd - 0.5;
                        const int k = (int)(g() % 5) - 2;
                        for (int q = 0; q < std::abs(k); ++q) x = std::nextafter(x, k > 0 ? 1.0 : -1.0);
                        break;
                    }
                    case 4: x = U(g) * 2000.0 - 1000.0; break;               // wrapped coordinates
                    default: {                                               // random significands
                        unsigned long long b = g();
                        b &= ~(0x7FFull << 52);
                        b |= (unsigned long long)(1023 - 1 - (g() % 12)) << 52;
                        std::memcpy(&x, &b, sizeof x);
                    }
                }
                volatile double xw = x - std::floor(x + 0.5);
                volatile double t = xw + 0.5;
                volatile double u = nd * t;
                volatile double v = u - alpha;
                volatile double l0 = std::ceil(v);
                volatile double s = l0 - v;
                ++total;
                long long l0i;
                double s2;
                if (!reduce_fixed(t, c, l0i, s2)) continue;
                ++fixed;
                const double sv = s;
                if ((double)l0i != l0 || std::memcmp(&sv, &s2, sizeof sv) != 0) {
                    if (bad < 5)
                        std::printf("mismatch L=%d m=%d x=%.17g l0=%.0f/%lld s=%.17g/%.17g\n", L, m, x, (double)l0,
                                    l0i, sv, s2);
                    ++bad;
                }
            }
        }
    std::printf("cases %lld fixed %lld mismatches %lld\n", total, fixed, bad);
    return bad != 0;
}
