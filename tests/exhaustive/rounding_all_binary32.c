/* Exhaustive check of the oracle's rounding (orc_round) over every finite
 * binary32 bit pattern (2^32 - 2^24 of them):
 *   to binary16 against the compiler's native _Float16 conversion (libgcc's
 *   soft-float routine on x86-64, the FCVT instruction on aarch64), value and
 *   sign, overflow to infinity and gradual underflow included;
 *   to bfloat16 against the round-to-nearest-even bit formula on the binary32
 *   encoding (add 0x7FFF plus the lowest kept bit, clear the low 16 bits).
 * Both references are independent of the oracle's scaling-based rounding.
 * Usage: rounding_all_binary32 <path to liboracle.so>; prints
 * "checked <n> fp16_mismatches <a> bf16_mismatches <b>". Test infrastructure. */
#include <dlfcn.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

typedef double (*round_fn)(double, int);

static int same(double a, double b) { return a == b && signbit(a) == signbit(b); }

int main(int argc, char **argv)
{
    if (argc < 2) return 2;
    void *lib = dlopen(argv[1], RTLD_NOW);
    if (!lib) { fprintf(stderr, "%s\n", dlerror()); return 2; }
    round_fn rnd = (round_fn)dlsym(lib, "orc_round");
    if (!rnd) return 2;
    long long checked = 0, bad16 = 0, badbf = 0;
#pragma omp parallel for schedule(static, 1 << 16) reduction(+ : checked, bad16, badbf)
    for (long long u = 0; u < (1LL << 32); u++) {
        const uint32_t b = (uint32_t)u;
        if ((b & 0x7F800000u) == 0x7F800000u) continue; /* inf / NaN */
        float f;
        memcpy(&f, &b, 4);
        const double x = (double)f;
        checked++;
        const _Float16 h = (_Float16)f;
        if (!same(rnd(x, 2), (double)h)) bad16++;
        uint32_t r = (b + 0x7FFFu + ((b >> 16) & 1u)) & 0xFFFF0000u;
        float fb;
        memcpy(&fb, &r, 4);
        if (!same(rnd(x, 3), (double)fb)) badbf++;
    }
    printf("checked %lld fp16_mismatches %lld bf16_mismatches %lld\n", checked, bad16, badbf);
    return 0;
}
