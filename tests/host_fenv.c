/* Host binary32 arithmetic under a chosen IEEE rounding direction.
 * Test pin for the 1/8/23 format (the paper's FP32, Sec. 5.2): the host FPU
 * computes a correctly rounded binary32 sum, product or quotient in round-to-nearest-even
 * or round-toward-zero.  Built by the tests with -frounding-math
 * -ffp-contract=off; no flush-to-zero is enabled. */
#include <fenv.h>
#include <stdint.h>
#include <string.h>

#pragma STDC FENV_ACCESS ON

static float as_f(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint32_t as_u(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

/* op: 0 add, 1 mul, 2 div; rz: 0 = FE_TONEAREST, 1 = FE_TOWARDZERO */
void host_f32(int op, int rz, const uint32_t *a, const uint32_t *b, uint32_t *out, long n) {
    int old = fegetround();
    fesetround(rz ? FE_TOWARDZERO : FE_TONEAREST);
    for (long i = 0; i < n; i++) {
        volatile float x = as_f(a[i]), y = as_f(b[i]);
        volatile float r = op == 0 ? x + y : (op == 1 ? x * y : x / y);
        out[i] = as_u(r);
    }
    fesetround(old);
}
