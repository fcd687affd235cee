/* Exhaustive check of the oracle's correctly rounded a + b and a * b in
 * binary16 or bfloat16 (orc_op_array) over every pair of finite operands of
 * the format (a - b is a + (-b) and is covered by the sign of b), against
 * references computed in binary32 and rounded by independent routines: the
 * compiler's _Float16 conversion for binary16, the round-to-nearest-even bit
 * formula for bfloat16. binary32 holds at least 2p + 2 bits for both formats,
 * so rounding its result once more is innocuous (the double-rounding theorem)
 * and the references are correctly rounded.
 * Usage: ops_all_pairs <path to liboracle.so> <fmt 2|3> <op 0 add|2 mul>;
 * prints "pairs <n> mismatches <m>". Test infrastructure. */
#include <dlfcn.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef void (*op_array_fn)(int64_t, int, const double *, const double *, int, double *);

static double bf16_value(uint16_t u) { uint32_t b = (uint32_t)u << 16; float f; memcpy(&f, &b, 4); return f; }
static double rne_bf16(float f)
{
    uint32_t b;
    memcpy(&b, &f, 4);
    if ((b & 0x7F800000u) == 0x7F800000u) return f; /* inf stays inf */
    b = (b + 0x7FFFu + ((b >> 16) & 1u)) & 0xFFFF0000u;
    float r;
    memcpy(&r, &b, 4);
    return r;
}
static int same(double a, double b) { return (a == b && signbit(a) == signbit(b)) || (isnan(a) && isnan(b)); }

int main(int argc, char **argv)
{
    if (argc < 4) return 2;
    void *lib = dlopen(argv[1], RTLD_NOW);
    if (!lib) { fprintf(stderr, "%s\n", dlerror()); return 2; }
    op_array_fn opf = (op_array_fn)dlsym(lib, "orc_op_array");
    const int fmt = atoi(argv[2]), op = atoi(argv[3]);
    if (!opf || (fmt != 2 && fmt != 3) || (op != 0 && op != 2)) return 2;
    /* every finite value of the format */
    static double vals[65536];
    int nv = 0;
    for (int u = 0; u < 65536; u++) {
        double v;
        if (fmt == 2) {
            _Float16 h;
            uint16_t s = (uint16_t)u;
            memcpy(&h, &s, 2);
            v = (double)h;
        } else {
            v = bf16_value((uint16_t)u);
        }
        if (isfinite(v)) vals[nv++] = v;
    }
    long long pairs = 0, bad = 0;
#pragma omp parallel reduction(+ : pairs, bad)
    {
        double *A = malloc(sizeof(double) * nv), *R = malloc(sizeof(double) * nv);
#pragma omp for schedule(dynamic, 64)
        for (int i = 0; i < nv; i++) {
            for (int j = 0; j < nv; j++) A[j] = vals[i];
            opf(nv, op, A, vals, fmt, R);
            const float fa = (float)vals[i];
            for (int j = 0; j < nv; j++) {
                const float fb = (float)vals[j];
                const float r32 = op == 0 ? fa + fb : fa * fb;
                const double ref = fmt == 2 ? (double)(_Float16)r32 : rne_bf16(r32);
                if (!same(R[j], ref)) bad++;
            }
            pairs += nv;
        }
        free(A);
        free(R);
    }
    printf("pairs %lld mismatches %lld\n", pairs, bad);
    return 0;
}
