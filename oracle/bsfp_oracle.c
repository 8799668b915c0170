/*
 * bsfp_oracle.c -- plain, slow, obviously-correct CPU oracle for bitslice
 * custom-precision floating point (Xu & Gregg, "Customizable Precision of
 * Floating-Point Arithmetic with Bitslice Vector Types", arXiv 1602.04716).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this code.  The product
 * path (the CUDA library) shares no code with it and never calls it.
 *
 * What it computes (the plain definition, not a circuit):
 *   every finite value of format 1/E/M is (-1)^s * Mant * 2^q with an integer
 *   significand Mant < 2^(M+1); an operation forms the EXACT result with
 *   arbitrary-precision integers, then rounds it once, either to nearest with
 *   ties to even (RN) or toward zero (RZ) -- the two rounding modes of the
 *   paper's Sec. 4.  The paper follows "the classic implementation of floating
 *   arithmetic in hardware" (Sec. 4) and is silent on bias, subnormals,
 *   Inf/NaN, overflow and the sign of zero; this oracle takes the IEEE-754
 *   reading for each (bias 2^(E-1)-1, gradual underflow, Inf/NaN at the
 *   all-ones exponent, RN overflow to Inf, RZ overflow to the largest finite
 *   value, x+(-x) = +0, canonical NaN = sign 0, exponent all ones, fraction
 *   1<<(M-1)).
 *
 *   Flush to zero (an optional mode, not in the paper): an operand with
 *   exponent field 0 is read as a zero of its sign, and a nonzero exact result
 *   whose magnitude is below the smallest normal 2^(1-bias) is a zero of its
 *   sign (tininess judged on the exact value, before rounding); everything
 *   else is rounded as above with M+1 significant bits.
 *
 *   pack / unpack follow the bitslice layout of Sec. 2 (Fig. 1) and Sec. 4
 *   (Fig. 3): bit b of element i lives in bit (i mod 32) of word i/32 of slice
 *   b; slice 0 is the least significant bit of the encoding (the carry of the
 *   Fig. 2 adder runs from slice i to slice i+1).
 *
 * Nothing here is blocked, fused or reordered beyond the definition.  The
 * element loops carry an OpenMP pragma only so that a timed baseline can use
 * the host's cores; each element is computed independently.
 */
#include <stdint.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* A fixed 320-bit unsigned integer: enough for any exact sum of two finite  */
/* values of a format with E <= 8, M <= 23 (at most 2^8 + 24 bits).           */
/* ------------------------------------------------------------------------ */
#define NLIMB 5
typedef struct { uint64_t w[NLIMB]; } big;

static void big_zero(big *a) { memset(a, 0, sizeof *a); }

static void big_from_u64(big *a, uint64_t v) { big_zero(a); a->w[0] = v; }

static int big_is_zero(const big *a) {
    for (int i = 0; i < NLIMB; i++) if (a->w[i]) return 0;
    return 1;
}

/* a <<= s, 0 <= s < 64*NLIMB; bits shifted past the top are lost (callers
 * never shift that far). */
static void big_shl(big *a, int s) {
    big r; big_zero(&r);
    int limb = s / 64, bit = s % 64;
    for (int i = NLIMB - 1; i >= 0; i--) {
        int src = i - limb;
        if (src < 0) continue;
        uint64_t v = a->w[src] << bit;
        if (bit && src - 1 >= 0) v |= a->w[src - 1] >> (64 - bit);
        r.w[i] = v;
    }
    *a = r;
}

/* r = a >> s (floor), s >= 0 */
static void big_shr(big *r, const big *a, int s) {
    big t; big_zero(&t);
    if (s >= 64 * NLIMB) { *r = t; return; }
    int limb = s / 64, bit = s % 64;
    for (int i = 0; i < NLIMB; i++) {
        int src = i + limb;
        if (src >= NLIMB) break;
        uint64_t v = a->w[src] >> bit;
        if (bit && src + 1 < NLIMB) v |= a->w[src + 1] << (64 - bit);
        t.w[i] = v;
    }
    *r = t;
}

static int big_cmp(const big *a, const big *b) {
    for (int i = NLIMB - 1; i >= 0; i--) {
        if (a->w[i] < b->w[i]) return -1;
        if (a->w[i] > b->w[i]) return 1;
    }
    return 0;
}

static void big_add(big *r, const big *a, const big *b) {
    uint64_t c = 0;
    for (int i = 0; i < NLIMB; i++) {
        uint64_t s = a->w[i] + c;
        uint64_t c1 = s < c;
        uint64_t t = s + b->w[i];
        c = c1 + (t < s);
        r->w[i] = t;
    }
}

/* r = a - b, requires a >= b */
static void big_sub(big *r, const big *a, const big *b) {
    uint64_t br = 0;
    for (int i = 0; i < NLIMB; i++) {
        uint64_t t = a->w[i] - b->w[i];
        uint64_t b1 = a->w[i] < b->w[i];
        uint64_t u = t - br;
        uint64_t b2 = t < br;
        r->w[i] = u;
        br = b1 | b2;
    }
}

/* number of significant bits (0 for zero) */
static int big_bitlen(const big *a) {
    for (int i = NLIMB - 1; i >= 0; i--)
        if (a->w[i]) return 64 * i + 64 - __builtin_clzll(a->w[i]);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Format                                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int E, M, rz, ftz;     /* exponent bits, fraction bits, 1 = round toward zero, 1 = flush to zero */
    int bias, emax;        /* bias = 2^(E-1)-1, emax = 2^E-1 (all-ones field)      */
} fmt_t;

/* mode: bit 0 = round toward zero (else to nearest even), bit 1 = flush to zero */
static fmt_t mkfmt(int E, int M, int mode) {
    fmt_t f;
    f.E = E; f.M = M; f.rz = mode & 1; f.ftz = (mode >> 1) & 1;
    f.bias = (1 << (E - 1)) - 1;
    f.emax = (1 << E) - 1;
    return f;
}

enum { CLS_FINITE = 0, CLS_INF = 1, CLS_NAN = 2 };

typedef struct {
    int cls;
    int s;            /* sign */
    uint64_t mant;    /* integer significand, < 2^(M+1); 0 for zero */
    int q;            /* value = (-1)^s * mant * 2^q */
} val_t;

/* Decode a B-bit pattern (bits above B ignored). */
static val_t decode(const fmt_t *f, uint32_t x) {
    val_t v;
    uint32_t frac = x & ((1u << f->M) - 1u);
    uint32_t e = (x >> f->M) & (uint32_t)f->emax;
    v.s = (int)((x >> (f->M + f->E)) & 1u);
    if ((int)e == f->emax) {
        v.cls = frac ? CLS_NAN : CLS_INF;
        v.mant = 0; v.q = 0;
        return v;
    }
    v.cls = CLS_FINITE;
    if (e == 0) {                       /* zero or subnormal (zero when flushing) */
        v.mant = f->ftz ? 0 : frac;
        v.q = 1 - f->bias - f->M;
    } else {                            /* normal: implicit leading one */
        v.mant = ((uint64_t)1 << f->M) + frac;
        v.q = (int)e - f->bias - f->M;
    }
    return v;
}

static uint32_t enc(const fmt_t *f, int s, uint32_t e, uint32_t frac) {
    return ((uint32_t)s << (f->E + f->M)) | (e << f->M) | frac;
}

static uint32_t canonical_nan(const fmt_t *f) {
    return enc(f, 0, (uint32_t)f->emax, 1u << (f->M - 1));
}

static uint32_t infinity(const fmt_t *f, int s) { return enc(f, s, (uint32_t)f->emax, 0); }

static uint32_t max_finite(const fmt_t *f, int s) {
    return enc(f, s, (uint32_t)f->emax - 1u, (1u << f->M) - 1u);
}

/* Round the exact nonzero value (-1)^s * T * 2^q to the format (RN-even or RZ)
 * and encode it.  This is the single rounding every operation ends with. */
static uint32_t round_encode(const fmt_t *f, int s, const big *T, int q) {
    const int M = f->M;
    int k = big_bitlen(T);                 /* T >= 1 */
    int u = k - 1 + q;                     /* exponent of the leading bit */
    int qmin = 1 - f->bias - M;            /* weight of the smallest subnormal */
    int r;                                 /* number of low bits dropped */
    if (f->ftz && u < 1 - f->bias)         /* tiny: a zero of the result's sign */
        return enc(f, s, 0, 0);
    if (u >= 1 - f->bias) r = k - (M + 1); /* normal range: keep M+1 bits */
    else r = qmin - q;                     /* subnormal range: quantise to 2^qmin */

    uint64_t Tp;
    if (r <= 0) {
        big t = *T;
        big_shl(&t, -r);
        Tp = t.w[0];                       /* exact; fits in M+1 bits */
    } else {
        big t;
        big_shr(&t, T, r);
        Tp = t.w[0];
        if (!f->rz) {
            /* remainder = T - (Tp << r), compared with half = 2^(r-1) */
            big back = t, rem, half;
            big_shl(&back, r);
            big_sub(&rem, T, &back);
            big_from_u64(&half, 1);
            big_shl(&half, r - 1);
            int c = big_cmp(&rem, &half);
            if (c > 0 || (c == 0 && (Tp & 1u))) Tp += 1;
        }
    }
    int qp = q + r;
    if (Tp == ((uint64_t)1 << (M + 1))) { Tp >>= 1; qp += 1; }  /* rounding carried out */

    long e; uint32_t frac;
    if (Tp >= ((uint64_t)1 << M)) { e = (long)qp + M + f->bias; frac = (uint32_t)(Tp - ((uint64_t)1 << M)); }
    else { e = 0; frac = (uint32_t)Tp; }

    if (e >= f->emax)                      /* overflow */
        return f->rz ? max_finite(f, s) : infinity(f, s);
    return enc(f, s, (uint32_t)e, frac);
}

/* x + y, one rounding. */
static uint32_t o_add(const fmt_t *f, uint32_t x, uint32_t y) {
    val_t a = decode(f, x), b = decode(f, y);
    if (a.cls == CLS_NAN || b.cls == CLS_NAN) return canonical_nan(f);
    if (a.cls == CLS_INF && b.cls == CLS_INF)
        return (a.s == b.s) ? infinity(f, a.s) : canonical_nan(f);
    if (a.cls == CLS_INF) return infinity(f, a.s);
    if (b.cls == CLS_INF) return infinity(f, b.s);

    /* exact sum at the common exponent q0 = min(qa, qb) */
    int q0 = a.q < b.q ? a.q : b.q;
    big A, Bv;
    big_from_u64(&A, a.mant);  big_shl(&A, a.q - q0);
    big_from_u64(&Bv, b.mant); big_shl(&Bv, b.q - q0);
    big T; int s;
    if (a.s == b.s) { big_add(&T, &A, &Bv); s = a.s; }
    else {
        int c = big_cmp(&A, &Bv);
        if (c >= 0) { big_sub(&T, &A, &Bv); s = a.s; }
        else        { big_sub(&T, &Bv, &A); s = b.s; }
    }
    if (big_is_zero(&T))               /* exact zero: +0 unless both are -0 */
        return enc(f, (a.s && b.s) ? 1 : 0, 0, 0);
    return round_encode(f, s, &T, q0);
}

/* x * y, one rounding. */
static uint32_t o_mul(const fmt_t *f, uint32_t x, uint32_t y) {
    val_t a = decode(f, x), b = decode(f, y);
    int s = a.s ^ b.s;
    if (a.cls == CLS_NAN || b.cls == CLS_NAN) return canonical_nan(f);
    if (a.cls == CLS_INF || b.cls == CLS_INF) {
        int other_zero = (a.cls == CLS_FINITE && a.mant == 0) || (b.cls == CLS_FINITE && b.mant == 0);
        return other_zero ? canonical_nan(f) : infinity(f, s);
    }
    uint64_t P = a.mant * b.mant;      /* < 2^48 */
    if (P == 0) return enc(f, s, 0, 0);
    big T; big_from_u64(&T, P);
    return round_encode(f, s, &T, a.q + b.q);
}

/* x / y, one rounding (the division of Sec. 4, Table 1).  IEEE-754 cases:
 * NaN for a NaN operand, 0/0 and Inf/Inf; x/0 = Inf and x/Inf = 0 with the
 * sign of x*y.  Otherwise the exact quotient mant_x / mant_y * 2^(qx - qy)
 * becomes T * 2^q with K = 2M + 8 extra quotient bits, whose lowest bit is
 * set when the division leaves a remainder: T has at least M + 9 bits, so
 * that bit lies at least seven places below the rounding position and only
 * records "inexact", which is all that rounding needs from the bits below. */
static uint32_t o_div(const fmt_t *f, uint32_t x, uint32_t y) {
    val_t a = decode(f, x), b = decode(f, y);
    int s = a.s ^ b.s;
    if (a.cls == CLS_NAN || b.cls == CLS_NAN) return canonical_nan(f);
    if (a.cls == CLS_INF) return b.cls == CLS_INF ? canonical_nan(f) : infinity(f, s);
    if (b.cls == CLS_INF) return enc(f, s, 0, 0);
    if (b.mant == 0) return a.mant == 0 ? canonical_nan(f) : infinity(f, s);
    if (a.mant == 0) return enc(f, s, 0, 0);
    const int K = 2 * f->M + 8;                      /* <= 54: the numerator fits in 128 bits */
    unsigned __int128 num = (unsigned __int128)a.mant << K;
    unsigned __int128 quo = num / b.mant, rem = num % b.mant;
    quo = (quo << 1) | (rem != 0);
    big T; big_zero(&T);
    T.w[0] = (uint64_t)quo;
    T.w[1] = (uint64_t)(quo >> 64);
    return round_encode(f, s, &T, a.q - b.q - K - 1);
}

static uint32_t flip_sign(const fmt_t *f, uint32_t y) { return y ^ (1u << (f->E + f->M)); }

/* ------------------------------------------------------------------------ */
/* Exported element-wise entry points (ctypes).  rz: the rounding mode,     */
/* 0 = RN-even, 1 = RZ, 2 = RN with flush to zero, 3 = RZ with flush.      */
/* ------------------------------------------------------------------------ */
uint32_t oracle_add1(int E, int M, int rz, uint32_t x, uint32_t y) { fmt_t f = mkfmt(E, M, rz); return o_add(&f, x, y); }
uint32_t oracle_sub1(int E, int M, int rz, uint32_t x, uint32_t y) { fmt_t f = mkfmt(E, M, rz); return o_add(&f, x, flip_sign(&f, y)); }
uint32_t oracle_mul1(int E, int M, int rz, uint32_t x, uint32_t y) { fmt_t f = mkfmt(E, M, rz); return o_mul(&f, x, y); }
uint32_t oracle_div1(int E, int M, int rz, uint32_t x, uint32_t y) { fmt_t f = mkfmt(E, M, rz); return o_div(&f, x, y); }
uint32_t oracle_fma2_1(int E, int M, int rz, uint32_t x, uint32_t y, uint32_t z) {
    fmt_t f = mkfmt(E, M, rz);
    return o_add(&f, o_mul(&f, x, y), z);
}

/* op: 0 add, 1 sub, 2 mul, 3 fma2 (a*b rounded, then + c rounded), 4 div */
void oracle_binop(int op, int E, int M, int rz, const uint32_t *a, const uint32_t *b,
                  const uint32_t *c, uint32_t *out, int64_t n) {
    fmt_t f = mkfmt(E, M, rz);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        uint32_t r;
        switch (op) {
        case 0: r = o_add(&f, a[i], b[i]); break;
        case 1: r = o_add(&f, a[i], flip_sign(&f, b[i])); break;
        case 2: r = o_mul(&f, a[i], b[i]); break;
        case 4: r = o_div(&f, a[i], b[i]); break;
        default: r = o_add(&f, o_mul(&f, a[i], b[i]), c[i]); break;
        }
        out[i] = r;
    }
}

/* Conversion from IEEE binary32 (the paper's FP32, Sec. 5.2) to 1/E/M: the
 * exact value of the binary32 encoding, rounded once in the target's mode
 * (NaN -> the canonical NaN, infinities and zeros keep their sign).  A
 * binary32 subnormal is an ordinary (tiny) value here; under flush to zero
 * it becomes a zero like any other tiny result. */
static uint32_t o_from_f32(const fmt_t *f, uint32_t x) {
    fmt_t f32 = mkfmt(8, 23, 0);
    val_t v = decode(&f32, x);
    if (v.cls == CLS_NAN) return canonical_nan(f);
    if (v.cls == CLS_INF) return infinity(f, v.s);
    if (v.mant == 0) return enc(f, v.s, 0, 0);
    big T; big_from_u64(&T, v.mant);
    return round_encode(f, v.s, &T, v.q);
}

/* Conversion from 1/E/M to binary32: exact (E <= 8, M <= 23), operands read
 * under the format's mode (flush to zero reads exponent field 0 as zero). */
static uint32_t o_to_f32(const fmt_t *f, uint32_t x) {
    fmt_t f32 = mkfmt(8, 23, 0);
    val_t v = decode(f, x);
    if (v.cls == CLS_NAN) return canonical_nan(&f32);
    if (v.cls == CLS_INF) return infinity(&f32, v.s);
    if (v.mant == 0) return enc(&f32, v.s, 0, 0);
    big T; big_from_u64(&T, v.mant);
    return round_encode(&f32, v.s, &T, v.q);
}

void oracle_from_f32(int E, int M, int mode, const uint32_t *x, uint32_t *out, int64_t n) {
    fmt_t f = mkfmt(E, M, mode);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) out[i] = o_from_f32(&f, x[i]);
}

void oracle_to_f32(int E, int M, int mode, const uint32_t *x, uint32_t *out, int64_t n) {
    fmt_t f = mkfmt(E, M, mode);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) out[i] = o_to_f32(&f, x[i]);
}

/* Integer bitslice vectors (Sec. 3, Fig. 2): elements are w-bit unsigned
 * integers (1 <= w <= 32); add, sub and mul keep the low w bits of the exact
 * result, i.e. arithmetic modulo 2^w (the carry out of the top slice is
 * dropped, as in the Fig. 2 adder).  op: 0 add, 1 sub, 2 mul. */
void oracle_int_binop(int op, int w, const uint32_t *a, const uint32_t *b, uint32_t *out, int64_t n) {
    const uint64_t mask = (w >= 32) ? 0xFFFFFFFFull : ((1ull << w) - 1ull);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        const uint64_t x = a[i] & mask, y = b[i] & mask;
        uint64_t r;
        switch (op) {
        case 0: r = x + y; break;
        case 1: r = x + ((mask + 1ull) - y); break;   /* x - y modulo 2^w */
        default: r = x * y; break;
        }
        out[i] = (uint32_t)(r & mask);
    }
}

/* Bitslice plane stride in 32-bit words: ceil(n/32) rounded up to 32 words. */
int64_t oracle_plane_stride(int64_t n) {
    int64_t words = (n + 31) / 32;
    return (words + 31) / 32 * 32;
}

/* pack: bit b of x[i] -> bit (i % 32) of planes[b*S + i/32]; everything else 0. */
void oracle_pack(int B, const uint32_t *x, int64_t n, uint32_t *planes, int64_t S) {
    memset(planes, 0, sizeof(uint32_t) * (size_t)B * (size_t)S);
    for (int64_t i = 0; i < n; i++)
        for (int b = 0; b < B; b++)
            if ((x[i] >> b) & 1u)
                planes[(int64_t)b * S + i / 32] |= 1u << (i % 32);
}

/* unpack: inverse of pack. */
void oracle_unpack(int B, const uint32_t *planes, int64_t S, int64_t n, uint32_t *x) {
    for (int64_t i = 0; i < n; i++) {
        uint32_t v = 0;
        for (int b = 0; b < B; b++)
            v |= ((planes[(int64_t)b * S + i / 32] >> (i % 32)) & 1u) << b;
        x[i] = v;
    }
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads for the following calls (the CPU baseline is timed at one core
 * and at all cores); k <= 0 is ignored. */
void oracle_set_threads(int k) {
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}
