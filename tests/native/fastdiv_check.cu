// Host-only check of the library's division by invariant integers against
// plain integer division: exhaustive over small numerators and random large
// ones, for every divisor the lattices use and a sweep of others.
#include <cstdio>
#include <cstdint>
#include "../../paper_1007_3432_gb300/csrc/hh_device.cuh"

int main()
{
    uint64_t state = 0x9E3779B97F4A7C15ull;
    auto next = [&]() {
        state ^= state << 13;
        state ^= state >> 7;
        state ^= state << 17;
        return state;
    };
    long long bad = 0, checked = 0;
    for (uint32_t d = 1; d <= 70000; d = d < 4200 ? d + 1 : d + 97) {
        hh::FastDiv f = hh::make_fastdiv(d);
        for (uint32_t n = 0; n < 5000; ++n, ++checked)
            if (hh::fd_div(n, f) != n / d) ++bad;
        for (int k = 0; k < 2000; ++k, ++checked) {
            uint32_t n = (uint32_t)next();
            if (hh::fd_div(n, f) != n / d) ++bad;
        }
        uint32_t edge[] = {0xFFFFFFFFu, 0x7FFFFFFFu, 0x80000000u, d - 1, d, d + 1};
        for (uint32_t n : edge) {
            ++checked;
            if (hh::fd_div(n, f) != n / d) ++bad;
        }
    }
    uint32_t lattice_divisors[] = {2, 3, 8, 10, 12, 16, 20, 24, 32, 64, 1024, 2048, 512, 1000,
                                   1728, 4096, 8000, 13824, 32768};
    for (uint32_t d : lattice_divisors) {
        hh::FastDiv f = hh::make_fastdiv(d);
        for (uint32_t n = 0; n < 8000000; n += 3, ++checked)
            if (hh::fd_div(n, f) != n / d) ++bad;
    }
    printf("checked %lld bad %lld\n", checked, bad);
    return bad == 0 ? 0 : 1;
}
