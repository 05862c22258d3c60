// Prints the cost model's choice for a list of product sizes, one line per
// size: "na nb kind est_us" (kind 1 schoolbook, 2 one 64-bit prime, 3 two
// 64-bit primes, 4 three 32-bit primes).
#include <cstdio>

#include "bn_internal.h"

int main() {
    const unsigned sizes[][2] = {{1, 1},     {32, 32},     {64, 64},     {128, 128},   {256, 256},
                                 {512, 512}, {1024, 1024}, {2048, 2048}, {4096, 4096}, {8192, 8192},
                                 {8192, 1},  {8192, 64},   {3000, 5000}, {700, 300}};
    for (auto &s : sizes) {
        const bn::MulChoice c = bn::choose_mul(s[0], s[1]);
        std::printf("%u %u %u %.6f\n", s[0], s[1], c.kind, c.est_us);
    }
    return 0;
}
