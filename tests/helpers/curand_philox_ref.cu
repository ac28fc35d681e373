// Host-only driver around cuRAND's header implementation of Philox4x32-10,
// used as an independent library check of the oracle's generator.  Reads
// lines "c0 c1 c2 c3 k0 k1" (decimal) from stdin, prints the four output words.
#define QUALIFIERS static inline __host__ __device__
#include <curand_philox4x32_x.h>
#include <cstdio>

int main()
{
    unsigned c0, c1, c2, c3, k0, k1;
    while (std::scanf("%u %u %u %u %u %u", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
        uint4 c = {c0, c1, c2, c3};
        uint2 k = {k0, k1};
        uint4 o = curand_Philox4x32_10(c, k);
        std::printf("%u %u %u %u\n", o.x, o.y, o.z, o.w);
    }
    return 0;
}
