/*
 * circuit.cuh -- bitslice floating-point circuits (host + device templates).
 *
 * Xu & Gregg, "Customizable Precision of Floating-Point Arithmetic with
 * Bitslice Vector Types" (arXiv 1602.04716).
 *
 * A value of the format 1/E/M (one sign bit, E exponent bits with bias
 * 2^(E-1)-1, M fraction bits) is held as B = 1+E+M words, one word per bit
 * ("slice"): bit j of slice b is bit b of element j (Sec. 2, Fig. 1).  Slice 0
 * is the least significant fraction bit, slices M..M+E-1 the exponent,
 * slice B-1 the sign.  Every operation below is a straight-line logic circuit
 * over whole words, so one evaluation computes 32 elements at once (Sec. 3,
 * Fig. 2).
 *
 * The operations follow the step structure of Sec. 4, Table 1:
 *   add/sub : sign, alignment shift (log shifter, Sec. 4), significand add,
 *             normalisation (log shifter), rounding;
 *   mul     : sign, exponent add (the two exponent additions merged, Sec. 4),
 *             significand multiply (carry-save array kept in registers),
 *             normalisation, rounding.
 * Rounding is round-to-nearest-even (RN) or round-toward-zero (RZ), both
 * correctly rounded (Sec. 4).  Where the paper is silent the circuits take the
 * IEEE-754 reading: gradual underflow, Inf/NaN at the all-ones exponent,
 * canonical NaN = +, exponent all ones, fraction 1 << (M-1); RN overflow to
 * Inf and RZ overflow to the largest finite value; an exact-zero sum is +0
 * unless both addends are -0.
 *
 * Gate primitives.  The circuits use only the functions of <= 3 words below;
 * each compiles to a single LOP3 on sm_103a (a NOT is folded into the LOP3 that
 * consumes it).  Instantiated with another word type (see gatecount.cpp) the
 * same templates are counted gate by gate instead of evaluated.  The aim is the
 * one the paper states for its own circuits (Sec. 4): the fewest gates, not the
 * shortest latency -- 32 lanes x many warps supply the parallelism.
 */
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define BSFP_HD __host__ __device__ __forceinline__
#define BSFP_HDC __host__ __device__
#define BSFP_UNROLL _Pragma("unroll")
#else
#define BSFP_HD inline
#define BSFP_HDC
#define BSFP_UNROLL _Pragma("GCC unroll 128")
#endif

namespace bsfp {

/* ---------------------------------------------------------------- gates --- */
template <class W> BSFP_HD W NOT(W a) { return ~a; }
template <class W> BSFP_HD W AND(W a, W b) { return a & b; }
template <class W> BSFP_HD W OR(W a, W b) { return a | b; }
template <class W> BSFP_HD W XOR(W a, W b) { return a ^ b; }
template <class W> BSFP_HD W ANDN(W a, W b) { return a & ~b; }            /* a & !b        */
template <class W> BSFP_HD W XOR3(W a, W b, W c) { return a ^ b ^ c; }
template <class W> BSFP_HD W MAJ(W a, W b, W c) { return (a & b) | (c & (a | b)); }
template <class W> BSFP_HD W MUX(W s, W t, W f) { return (s & t) | (~s & f); } /* s ? t : f  */
template <class W> BSFP_HD W OR3(W a, W b, W c) { return a | b | c; }
template <class W> BSFP_HD W AND3(W a, W b, W c) { return a & b & c; }
template <class W> BSFP_HD W ANDOR(W a, W b, W c) { return (a & b) | c; }  /* a&b | c       */
template <class W> BSFP_HD W ANDNN(W a, W b, W c) { return a & ~b & ~c; }  /* a & !b & !c   */
/* The full-adder gates as single instructions: on the device, for 32-bit
 * words, XOR3 and MAJ are emitted as lop3.b32 with their truth tables, so the
 * compiler cannot regroup them (left to itself it may share x^y between the
 * sum and a majority rewritten as (x&y)|(z&(x^y)), which costs four
 * instructions per full adder instead of two).  Only for inputs that are
 * never constants: a constant input would no longer fold away. */
#if defined(__CUDA_ARCH__)
template <unsigned L>
__device__ __forceinline__ uint32_t lop3_hard(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(L));
    return d;
}
__device__ __forceinline__ uint32_t XOR3H(uint32_t a, uint32_t b, uint32_t c) { return lop3_hard<0x96u>(a, b, c); }
__device__ __forceinline__ uint32_t MAJH(uint32_t a, uint32_t b, uint32_t c) { return lop3_hard<0xE8u>(a, b, c); }
#endif
template <class W> BSFP_HD W XOR3H(W a, W b, W c) { return XOR3(a, b, c); }
template <class W> BSFP_HD W MAJH(W a, W b, W c) { return MAJ(a, b, c); }
/* Any function of three words, given by its truth table L: bit (4a+2b+c) of L
 * is the output for input bits a, b, c (the LOP3 immediate convention). */
template <unsigned L, class W> BSFP_HD W F3(W a, W b, W c) {
    W r = W(0u);
    if (L & 0x01u) r = r | (~a & ~b & ~c);
    if (L & 0x02u) r = r | (~a & ~b & c);
    if (L & 0x04u) r = r | (~a & b & ~c);
    if (L & 0x08u) r = r | (~a & b & c);
    if (L & 0x10u) r = r | (a & ~b & ~c);
    if (L & 0x20u) r = r | (a & ~b & c);
    if (L & 0x40u) r = r | (a & b & ~c);
    if (L & 0x80u) r = r | (a & b & c);
    return r;
}
/* Named truth tables used below. */
constexpr unsigned LUT_G_AND_LS = 0xE0u;     /* g & (l | s)          */
constexpr unsigned LUT_NZ_BUDGET = 0x0Bu;    /* !top & (!br | hiu)   */
constexpr unsigned LUT_OR_ANDN = 0x54u;      /* (m | o) & !s         */
constexpr unsigned LUT_ANDNN = 0x10u;        /* a & !b & !c          */
constexpr unsigned LUT_MASK_OR = 0xBAu;      /* (m & !z) | f         */
constexpr unsigned LUT_AND_OR_NOT = 0xD0u;   /* a & (b | !c)         */

/* -------------------------------------------------------- word vectors --- */
/* OR / AND of n words (n compile-time after inlining). */
template <int N, class W> BSFP_HD W or_n(const W* x) {
    if constexpr (N <= 0) {
        return W(0u);
    } else {
        W r = x[0];
        BSFP_UNROLL
        for (int i = 1; i < N; i += 2) r = (i + 1 < N) ? OR3(r, x[i], x[i + 1]) : OR(r, x[i]);
        return r;
    }
}
template <int N, class W> BSFP_HD W and_n(const W* x) {
    if constexpr (N <= 0) {
        return ~W(0u);
    } else {
        W r = x[0];
        BSFP_UNROLL
        for (int i = 1; i < N; i += 2) r = (i + 1 < N) ? AND3(r, x[i], x[i + 1]) : AND(r, x[i]);
        return r;
    }
}

/* One stage of a right log shifter: if dk, x >>= S, with every bit that falls
 * to position 0 or below ORed into x[0] (the sticky position). */
template <int N, int S, class W> BSFP_HD void rs_stage(W* x, W dk) {
    const W st = or_n<S>(x + 1);
    const W x0 = ANDOR(dk, st, x[0]);
    BSFP_UNROLL
    for (int p = 1; p < N; ++p) x[p] = MUX(dk, (p + S < N) ? x[(p + S < N) ? p + S : 0] : W(0u), x[p]);
    x[0] = x0;
}

/* x (N words, x[0] = sticky position) >>= d, d unsigned with ND bits (the log
 * shifter of Sec. 4).  Shift amounts >= N move every bit into the sticky. */
template <int N, int ND, int K = 0, class W> BSFP_HD void rshift_sticky(W* x, const W* d) {
    if constexpr (K < ND) {
        if constexpr ((1 << K) < N) {
            rs_stage<N, (1 << K)>(x, d[K]);
            rshift_sticky<N, ND, K + 1>(x, d);
        } else {
            const W far = or_n<ND - K>(d + K);
            const W st = or_n<N - 1>(x + 1);
            x[0] = ANDOR(far, st, x[0]);
            BSFP_UNROLL
            for (int p = 1; p < N; ++p) x[p] = ANDN(x[p], far);
        }
    }
}

BSFP_HDC constexpr int floor_log2(int v) { return v <= 1 ? 0 : 1 + floor_log2(v / 2); }

/* One stage of the normalising left shifter: shift by S = 2^K when the top S
 * bits of z are zero and the remaining budget allows it.  The budget test is
 * u >= (t[KT..K+1], 1, 0..0), i.e. u - (shift already taken) >= S, done as a
 * borrow chain over bits K..KT of u; hiu = some bit of u above KT is set. */
template <int N, int NU, int KT, int K, int LO, class W>
BSFP_HD void ln_stage(W* z, const W* u, W hiu, W* t, W* st) {
    constexpr int S = 1 << K;
    W c;
    if constexpr (K >= NU) {
        c = W(0u);                       /* budget < 2^NU <= S: never shift */
    } else {
        const W top = or_n<S>(z + N - S);
        W br = NOT(u[K]);
        BSFP_UNROLL
        for (int j = K + 1; j <= KT && j < NU; ++j) br = MAJ(NOT(u[j]), t[j], br);
        c = F3<LUT_NZ_BUDGET>(top, br, hiu);
    }
    t[K] = c;
    BSFP_UNROLL
    for (int p = N - 1; p >= 0; --p) z[p] = MUX(c, (p >= S) ? z[(p >= S) ? p - S : 0] : W(0u), z[p]);
    /* the later stages shift by at most S - 1 more, so a position p <= LO - S
     * ends below LO whatever they do: it only counts through the sticky OR.
     * Fold it into *st and clear it (bits only move up, so nothing above
     * depends on it), and the later stages' multiplexers on zeros vanish. */
    if constexpr (LO > 0) {
        BSFP_UNROLL
        for (int p = 0; p <= LO - S && p < N; ++p) {
            *st = OR(*st, z[p]);
            z[p] = W(0u);
        }
    }
}

template <int N, int NU, int KT, int K, int LO, class W>
BSFP_HD void ln_stages(W* z, const W* u, W hiu, W* t, W* st) {
    ln_stage<N, NU, KT, K, LO>(z, u, hiu, t, st);
    if constexpr (K > 0) ln_stages<N, NU, KT, K - 1, LO>(z, u, hiu, t, st);
}

/* Normalise z (N words, z[N-1] = top) left by t = min(lz(z), u) where u is an
 * unsigned NU-bit budget; writes the shift t[0..KT], KT = floor(log2(N-1)).
 * Greedy from the largest stage down: each stage removes 2^K leading zeros
 * when both the zeros and the budget allow, which decomposes min(lz, u)
 * exactly (the normalisation log shifter of Sec. 4, Table 1).
 * LO > 0: the caller uses positions below LO of the result only through
 * their OR (a sticky bit); they are OR-ed into *st (which the caller
 * initialises) as soon as no later stage can lift them to LO, and left
 * zero. */
template <int N, int NU, int LO = 0, class W> BSFP_HD void lnorm(W* z, const W* u, W* t, W* st = nullptr) {
    constexpr int KT = floor_log2(N - 1);
    W hiu = W(0u);
    if constexpr (KT + 1 < NU) hiu = or_n<NU - KT - 1>(u + KT + 1);
    ln_stages<N, NU, KT, KT, LO>(z, u, hiu, t, st);
}

/* D = u - t (u: NU bits, t: NT bits, u >= t), NU-bit result. */
template <int NU, int NT, class W> BSFP_HD void sub_un(const W* u, const W* t, W* D) {
    W br = W(0u);
    BSFP_UNROLL
    for (int i = 0; i < NU; ++i) {
        const W ti = (i < NT) ? t[(i < NT) ? i : 0] : W(0u);
        D[i] = XOR3(u[i], ti, br);
        if (i + 1 < NU) br = MAJ(NOT(u[i]), ti, br);
    }
}

/* mag = (D << M) + sig + rup, sig has M+1 bits (sig[M] = leading bit), D has
 * ND bits; mag has M+ND+1 bits.  Adding the leading bit into the exponent
 * field and the rounding carry through the whole magnitude is the usual
 * encoding trick: a fraction that rounds up from all ones increments the
 * exponent, and a subnormal that rounds up to 2^M becomes the least normal. */
template <int M, int ND, class W> BSFP_HD void assemble(const W* D, const W* sig, W rup, W* mag) {
    W c = rup;
    BSFP_UNROLL
    for (int i = 0; i < M; ++i) {
        mag[i] = XOR(sig[i], c);
        c = AND(sig[i], c);
    }
    mag[M] = XOR3(sig[M], D[0], c);
    c = MAJ(sig[M], D[0], c);
    BSFP_UNROLL
    for (int i = 1; i < ND; ++i) {
        mag[M + i] = XOR(D[i], c);
        c = AND(D[i], c);
    }
    mag[M + ND] = c;
}

/* Final encoding.  mag: M+NF bits (NF >= E field bits, higher ones only ever
 * signal overflow); spec: the result is Inf or NaN; nan: it is NaN; zero: the
 * exact result is zero (its exponent bits in mag are then meaningless, since
 * the normaliser cannot always shift a zero significand all the way down);
 * sgn: sign of the result unless zs (an exact zero that is +0).  RN overflows
 * to Inf, RZ to max finite. */
template <int E, int M, int NF, bool RZ, class W, bool FTZ = false>
BSFP_HD void encode(const W* mag_in, W spec, W nan, W zero, W sgn, W zs, W* r) {
    constexpr int B = 1 + E + M;
    /* with flush to zero a zero result may carry a nonzero significand (a
     * flushed tiny value): its fraction is cleared here */
    W mf[M + NF];
    BSFP_UNROLL
    for (int i = 0; i < M + NF; ++i) mf[i] = (FTZ && i < M) ? ANDN(mag_in[i], zero) : mag_in[i];
    const W* mag = mf;
    W ovf = and_n<E>(mag + M);
    if constexpr (NF > E) ovf = OR(ovf, or_n<NF - E>(mag + M + E));
    if constexpr (!RZ) {
        const W force = OR(ANDN(ovf, zero), spec);
        BSFP_UNROLL
        for (int i = 0; i < E; ++i) r[M + i] = F3<LUT_MASK_OR>(mag[M + i], zero, force);
        BSFP_UNROLL
        for (int i = 0; i + 1 < M; ++i) r[i] = ANDN(mag[i], force);
        r[M - 1] = MUX(force, nan, mag[M - 1]);
    } else {
        /* overflow -> exponent 2^E-2, fraction all ones; Inf/NaN -> all-ones
         * exponent with fraction 0 / 1 << (M-1) */
        const W ov = ANDN(ovf, zero);
        const W ovs = OR(ov, spec);
        r[M] = ANDOR(mag[M], NOT(OR(ovf, zero)), spec);
        BSFP_UNROLL
        for (int i = 1; i < E; ++i) r[M + i] = F3<LUT_MASK_OR>(mag[M + i], zero, ovs);
        BSFP_UNROLL
        for (int i = 0; i + 1 < M; ++i) r[i] = F3<LUT_OR_ANDN>(mag[i], ov, spec);
        r[M - 1] = MUX(spec, nan, OR(mag[M - 1], ov));
    }
    r[B - 1] = F3<LUT_ANDNN>(sgn, zs, nan);
}

/* -------------------------------------------------------------- add/sub --- */
/* r = a + b (NEG_B: a - b), one rounding (Sec. 4, Table 1, Add/Sub). */
template <int E, int M, bool RZ, bool NEG_B, bool FTZ = false, class W>
BSFP_HD void fp_add(const W* a, const W* b, W* r) {
    static_assert(E >= 2 && M >= 1 && 1 + E + M <= 32, "format out of range");
    constexpr int B = 1 + E + M;
    constexpr int NM = E + M;   /* magnitude bits */
    if constexpr (FTZ) {
        /* flush to zero: an operand with exponent field 0 is a zero of its
         * sign (its fraction is cleared); the sum of two such operands is
         * exact, so a tiny result is exactly a subnormal of the gradual-
         * underflow adder, and flushing it after the adder (fraction cleared
         * when the exponent field is 0) keeps the result's sign */
        W x[B], y[B];
        const W nza = or_n<E>(a + M), nzb = or_n<E>(b + M);
        BSFP_UNROLL
        for (int i = 0; i < B; ++i) {
            x[i] = i < M ? AND(a[i], nza) : a[i];
            y[i] = i < M ? AND(b[i], nzb) : b[i];
        }
        fp_add<E, M, RZ, NEG_B, false>(x, y, r);
        const W nzr = or_n<E>(r + M);
        BSFP_UNROLL
        for (int i = 0; i < M; ++i) r[i] = AND(r[i], nzr);
        return;
    }
    const W sa = a[B - 1];
    const W sb = NEG_B ? NOT(b[B - 1]) : b[B - 1];

    /* step 1 (sign): order the operands by magnitude, |X| >= |Y| -- a borrow
     * chain of |a| - |b| */
    W br = ANDN(b[0], a[0]);
    BSFP_UNROLL
    for (int i = 1; i < NM; ++i) br = MAJ(NOT(a[i]), b[i], br);
    const W sw = br;   /* |a| < |b| */
    W X[NM], Y[NM];
    BSFP_UNROLL
    for (int i = 0; i < NM; ++i) {
        X[i] = MUX(sw, b[i], a[i]);
        Y[i] = MUX(sw, a[i], b[i]);
    }
    const W sX = MUX(sw, sb, sa);
    const W esub = XOR(sa, sb);         /* effective subtraction */
    const W* eX = X + M;
    const W* eY = Y + M;
    const W nzX = or_n<E>(eX);          /* implicit bits: exponent field != 0 */
    const W nzY = or_n<E>(eY);

    /* exponent difference d = max(eX,1) - max(eY,1) >= 0 */
    W d[E];
    br = ANDN(nzX, nzY);
    BSFP_UNROLL
    for (int i = 0; i < E; ++i) {
        d[i] = XOR3(eX[i], eY[i], br);
        if (i + 1 < E) br = MAJ(NOT(eX[i]), eY[i], br);
    }

    /* step 2 (alignment shift): y = 1.fY (or 0.fY) at positions 3..M+3 above
     * guard (2), round (1) and sticky (0) */
    constexpr int NY = M + 4;
    W y[NY];
    y[0] = y[1] = y[2] = W(0u);
    BSFP_UNROLL
    for (int i = 0; i < M; ++i) y[3 + i] = Y[i];
    y[M + 3] = nzY;
    rshift_sticky<NY, E>(y, d);

    /* step 3 (add): z = x +/- y over M+5 positions (M+4 = carry out) */
    constexpr int NZ = M + 5;
    W z[NZ];
    W c = esub;
    BSFP_UNROLL
    for (int p = 0; p < NY; ++p) {
        const W xp = (p < 3) ? W(0u) : (p < M + 3 ? X[(p >= 3 && p < M + 3) ? p - 3 : 0] : nzX);
        const W yp = XOR(y[p], esub);
        z[p] = XOR3(xp, yp, c);
        c = MAJ(xp, yp, c);
    }
    z[NZ - 1] = ANDN(c, esub);

    /* step 4 (normalisation): shift left by t = min(lz(z), max(eX,1)); the
     * result exponent field is max(eX,1) + 1 - t, and a result that cannot be
     * normalised within that budget is subnormal */
    W u[E];
    u[0] = OR(eX[0], NOT(nzX));
    BSFP_UNROLL
    for (int i = 1; i < E; ++i) u[i] = eX[i];
    constexpr int KT = floor_log2(NZ - 1);
    W t[KT + 1];
    W stz = W(0u);                   /* sticky of the positions below the guard */
    lnorm<NZ, E, 3>(z, u, t, &stz);
    W D[E];
    sub_un<E, KT + 1>(u, t, D);

    /* step 5 (rounding): significand z[M+4..4], guard z[3], sticky z[2..0] */
    const W* sig = z + 4;
    W rup = W(0u);
    if constexpr (!RZ) rup = F3<LUT_G_AND_LS>(z[3], sig[0], OR(stz, OR3(z[2], z[1], z[0])));
    W mag[M + E + 1];
    assemble<M, E>(D, sig, rup, mag);

    /* specials: X is NaN or Inf whenever either operand is (|NaN| > |Inf|) */
    const W xspec = and_n<E>(eX);
    const W yspec = and_n<E>(eY);
    const W nan = AND(xspec, ANDOR(yspec, esub, or_n<M>(X)));
    const W zero = NOT(or_n<M + 1>(sig));            /* exact zero sum */
    const W zs = AND3(zero, esub, NOT(xspec));       /* x + (-x) = +0 */
    encode<E, M, E + 1, RZ>(mag, xspec, nan, zero, sX, zs, r);
}

/* ------------------------------------------------------------------ mul --- */
/* P = A * B for n-bit unsigned A, B (n >= 2): carry-save array, one row per
 * bit of B, then a ripple adder for the upper half (Sec. 4: the significand
 * product is unrolled and kept in registers).  After row j the sums S cover
 * columns 0..n+j-1 and the carries C columns j+1..j+n-1; the last cell of
 * every row has no sum or carry to add and passes its partial product
 * through, and row 1 has no carries yet (half adders), so every full adder
 * below has three variable inputs. */
template <int n, class W> BSFP_HD void umul(const W* A, const W* Bv, W* P) {
    W S[2 * n], C[2 * n];
    BSFP_UNROLL
    for (int i = 0; i < n; ++i) S[i] = AND(A[i], Bv[0]);
    BSFP_UNROLL
    for (int j = 1; j < n; ++j) {
        W nc[2 * n];
        BSFP_UNROLL
        for (int i = 0; i < n - 1; ++i) {
            const int w = i + j;
            const W pp = AND(A[i], Bv[j]);
            if (j == 1) {
                nc[w + 1] = AND(S[w], pp);
                S[w] = XOR(S[w], pp);
            } else {
                nc[w + 1] = MAJH(S[w], C[w], pp);
                S[w] = XOR3H(S[w], C[w], pp);
            }
        }
        S[n - 1 + j] = AND(A[n - 1], Bv[j]);
        BSFP_UNROLL
        for (int i = 0; i < n - 1; ++i) C[i + j + 1] = nc[i + j + 1];
    }
    BSFP_UNROLL
    for (int w = 0; w < n; ++w) P[w] = S[w];
    /* columns n..2n-2 hold S and C; column 2n-1 only the final carry */
    W c = AND(S[n], C[n]);
    P[n] = XOR(S[n], C[n]);
    BSFP_UNROLL
    for (int w = n + 1; w < 2 * n - 1; ++w) {
        P[w] = XOR3H(S[w], C[w], c);
        c = MAJH(S[w], C[w], c);
    }
    P[2 * n - 1] = c;
}

/* r = a * b with flush to zero: operands with exponent field 0 are zeros of
 * their sign, and a product whose exact magnitude is below the smallest
 * normal (tiny before rounding) is a zero of the product's sign.  Both
 * significands are then normal, the product lies in [1, 4) and needs a
 * one-position normalisation only: neither the leading-zero normaliser nor
 * the right shifter into the subnormal range of the gradual-underflow
 * multiplier is needed -- the gates the paper saves with a flush mode. */
template <int E, int M, bool RZ, class W> BSFP_HD void fp_mul_ftz(const W* a, const W* b, W* r) {
    constexpr int B = 1 + E + M;
    constexpr int N1 = M + 1;
    constexpr int NP = 2 * M + 2;
    constexpr int NU = E + 2;
    const W s = XOR(a[B - 1], b[B - 1]);
    const W* ea = a + M;
    const W* eb = b + M;
    const W nzA = or_n<E>(ea);
    const W nzB = or_n<E>(eb);

    /* significand product of 1.fa and 1.fb */
    W SA[N1], SB[N1];
    BSFP_UNROLL
    for (int i = 0; i < M; ++i) {
        SA[i] = a[i];
        SB[i] = b[i];
    }
    SA[M] = ~W(0u);
    SB[M] = ~W(0u);
    W P[NP];
    umul<N1>(SA, SB, P);
    const W top = P[NP - 1];

    /* D = ea + eb - bias - 1 + top in NU-bit two's complement (the exponent
     * field of the result is D + 1, the leading one being added by assemble):
     * a carry-save step of ea, eb and the constant -(bias + 1) = -2^(E-1),
     * then a ripple adder with top as carry-in */
    constexpr uint32_t KB = ((uint32_t)(-(1 << (E - 1)))) & ((1u << NU) - 1u);
    W D[NU];
    {
        W cs[NU], cc[NU + 1];
        cc[0] = W(0u);
        BSFP_UNROLL
        for (int i = 0; i < NU; ++i) {
            const W ai = (i < E) ? ea[(i < E) ? i : 0] : W(0u);
            const W bi = (i < E) ? eb[(i < E) ? i : 0] : W(0u);
            const bool k = (KB >> i) & 1u;
            cs[i] = k ? NOT(XOR(ai, bi)) : XOR(ai, bi);
            cc[i + 1] = k ? OR(ai, bi) : AND(ai, bi);
        }
        W c = top;
        BSFP_UNROLL
        for (int i = 0; i < NU; ++i) {
            D[i] = XOR3(cs[i], cc[i], c);
            if (i + 1 < NU) c = MAJ(cs[i], cc[i], c);
        }
    }
    const W tiny = D[NU - 1];        /* D < 0: exponent field < 1 */

    /* one-position normalisation, guard and sticky */
    W sig[N1];
    BSFP_UNROLL
    for (int i = 0; i < N1; ++i) sig[i] = MUX(top, P[M + 1 + i], P[M + i]);
    W rup = W(0u);
    if constexpr (!RZ) {
        const W g = MUX(top, P[M], P[M - 1 >= 0 ? M - 1 : 0]);
        const W st0 = or_n<M - 1>(P);                 /* below the guard when top = 0 */
        const W st = (M >= 1) ? ANDOR(top, P[M - 1], st0) : st0;
        rup = F3<LUT_G_AND_LS>(g, sig[0], st);
    }
    W mag[M + NU];
    assemble<M, NU - 1>(D, sig, rup, mag);

    /* specials: NaN for NaN operands and 0 * Inf (zeros include flushed
     * operands); Inf otherwise */
    const W aspec = and_n<E>(ea), bspec = and_n<E>(eb);
    const W fA = or_n<M>(a), fB = or_n<M>(b);
    const W nan = OR(F3<LUT_AND_OR_NOT>(aspec, fA, nzB), F3<LUT_AND_OR_NOT>(bspec, fB, nzA));
    const W zero = OR(NOT(AND(nzA, nzB)), tiny);
    encode<E, M, NU, RZ, W, true>(mag, OR(aspec, bspec), nan, zero, s, W(0u), r);
}

/* r = a * b, one rounding (Sec. 4, Table 1, Mul). */
template <int E, int M, bool RZ, bool FTZ = false, class W> BSFP_HD void fp_mul(const W* a, const W* b, W* r) {
    static_assert(E >= 2 && M >= 1 && 1 + E + M <= 32, "format out of range");
    if constexpr (FTZ) {
        fp_mul_ftz<E, M, RZ>(a, b, r);
        return;
    }
    constexpr int B = 1 + E + M;
    constexpr int N1 = M + 1;         /* significand bits */
    constexpr int NP = 2 * M + 2;     /* product bits */
    constexpr int NU = E + 2;         /* signed exponent sum */
    /* step 1: sign */
    const W s = XOR(a[B - 1], b[B - 1]);
    const W* ea = a + M;
    const W* eb = b + M;
    const W nzA = or_n<E>(ea);
    const W nzB = or_n<E>(eb);

    /* step 3: significand product */
    W SA[N1], SB[N1];
    BSFP_UNROLL
    for (int i = 0; i < M; ++i) {
        SA[i] = a[i];
        SB[i] = b[i];
    }
    SA[M] = nzA;
    SB[M] = nzB;
    W P[NP];
    umul<N1>(SA, SB, P);

    /* step 2: u = max(ea,1) + max(eb,1) - bias in NU-bit two's complement,
     * the two exponent additions merged into one carry-save step + one ripple
     * (Sec. 4).  u + 1 is the exponent field when the product's top bit
     * (position 2M+1) is set. */
    W ua[E], ub[E];
    ua[0] = OR(ea[0], NOT(nzA));
    ub[0] = OR(eb[0], NOT(nzB));
    BSFP_UNROLL
    for (int i = 1; i < E; ++i) {
        ua[i] = ea[i];
        ub[i] = eb[i];
    }
    constexpr uint32_t KB = (1u - (1u << (E - 1))) & ((1u << NU) - 1u);  /* -bias + ... : 1 - 2^(E-1) */
    W u[NU];
    {
        W cs[NU], cc[NU + 1];
        cc[0] = W(0u);
        BSFP_UNROLL
        for (int i = 0; i < NU; ++i) {
            const W ai = (i < E) ? ua[(i < E) ? i : 0] : W(0u);
            const W bi = (i < E) ? ub[(i < E) ? i : 0] : W(0u);
            const bool k = (KB >> i) & 1u;
            cs[i] = k ? NOT(XOR(ai, bi)) : XOR(ai, bi);
            cc[i + 1] = k ? OR(ai, bi) : AND(ai, bi);
        }
        W c = W(0u);
        BSFP_UNROLL
        for (int i = 0; i < NU; ++i) {
            u[i] = XOR3(cs[i], cc[i], c);
            if (i + 1 < NU) c = MAJ(cs[i], cc[i], c);
        }
    }
    const W neg = u[NU - 1];   /* u < 0: the product is below the normal range */

    /* step 4a (u >= 0): normalise left by t = min(lz(P), u) */
    W zl[NP];
    BSFP_UNROLL
    for (int i = 0; i < NP; ++i) zl[i] = P[i];
    W um[NU - 1];
    BSFP_UNROLL
    for (int i = 0; i < NU - 1; ++i) um[i] = ANDN(u[i], neg);    /* budget 0 when u < 0 */
    constexpr int KT = floor_log2(NP - 1);
    W t[KT + 1];
    W stl = W(0u);                   /* sticky of the positions below the guard zl[M] */
    lnorm<NP, NU - 1, M>(zl, um, t, &stl);
    W D[NU - 1];
    sub_un<NU - 1, KT + 1>(um, t, D);

    /* step 4b (u < 0): shift right by -u = ~u + 1 with sticky; the top M+2
     * product bits plus a sticky of the rest suffice.  q[0] sticky, q[1]
     * guard, q[2..M+2] significand, after the fixed shift by one. */
    constexpr int NQ = M + 3;
    W q[NQ];
    q[0] = or_n<M + 1>(P);
    BSFP_UNROLL
    for (int p = 1; p < NQ - 1; ++p) q[p] = P[M + p];
    q[NQ - 1] = W(0u);
    if constexpr (E >= 3) {
        W nu[E - 1];
        BSFP_UNROLL
        for (int i = 0; i < E - 1; ++i) nu[i] = NOT(u[i]);
        rshift_sticky<NQ, E - 1>(q, nu);
    }

    /* merge the two paths: significand, guard, sticky */
    W sig[N1];
    BSFP_UNROLL
    for (int i = 0; i < N1; ++i) sig[i] = MUX(neg, q[2 + i], zl[M + 1 + i]);
    W rup = W(0u);
    if constexpr (!RZ) {
        const W g = MUX(neg, q[1], zl[M]);
        const W st = MUX(neg, q[0], OR(stl, or_n<M>(zl)));
        rup = F3<LUT_G_AND_LS>(g, sig[0], st);
    }

    /* step 5: rounding into the encoded magnitude */
    W mag[M + NU];
    assemble<M, NU - 1>(D, sig, rup, mag);

    /* specials: NaN for NaN operands and 0 * Inf; Inf otherwise */
    const W aspec = and_n<E>(ea), bspec = and_n<E>(eb);
    const W fA = or_n<M>(a), fB = or_n<M>(b);
    const W tA = OR(nzA, fA), tB = OR(nzB, fB);     /* operand is nonzero */
    const W nan = OR(F3<LUT_AND_OR_NOT>(aspec, fA, tB), F3<LUT_AND_OR_NOT>(bspec, fB, tA));
    const W zero = NOT(AND(tA, tB));
    encode<E, M, NU, RZ>(mag, OR(aspec, bspec), nan, zero, s, W(0u), r);
}

/* ------------------------------------------------------------------ div --- */
BSFP_HDC constexpr int bit_length(int v) { return v <= 0 ? 0 : 1 + bit_length(v >> 1); }

/* r = a / b, one rounding (Sec. 4, Table 1, Div: restoring division).
 * 1. Both significands (implicit bit included) are normalised left by the
 *    log shifter, so that a subnormal operand has its leading one on top;
 *    the exponents become max(e,1) - shift.
 * 2. Restoring division: M+3 quotient bits of X / Y, most significant first,
 *    each a borrow chain R - Y (the bit is 1 when nothing is borrowed) and a
 *    multiplexer keeping R or R - Y, then a doubling of R; the final R != 0
 *    is the sticky bit.
 * 3. X / Y lies in (1/2, 2): the first quotient bit selects a one-position
 *    normalisation; the exponent field before rounding is
 *    ex' - ey' + bias - 1 + (first bit).
 * 4. Below the normal range the significand, guard and sticky shift right
 *    into the subnormal positions (a fixed shift by one, then the log
 *    shifter by the complement of the exponent), as in the multiplier.
 * 5. Rounding, overflow and the IEEE cases: NaN for NaN operands, 0/0 and
 *    Inf/Inf; x/0 and Inf/y are infinities, 0/y and x/Inf zeros, the sign
 *    the XOR of the signs.
 * With flush to zero the operands are normal or zero, step 1 and step 4
 * disappear, and a result below the normal range is a zero of its sign. */
template <int E, int M, bool RZ, bool FTZ = false, class W> BSFP_HD void fp_div(const W* a, const W* b, W* r) {
    static_assert(E >= 2 && M >= 1 && 1 + E + M <= 32, "format out of range");
    constexpr int B = 1 + E + M;
    constexpr int N1 = M + 1;
    constexpr int KT = floor_log2(N1 - 1);                           /* shift counts have KT+1 bits */
    constexpr int NU = bit_length((1 << (E + 1)) + 2 * M + 16) + 1;  /* signed exponent width */
    constexpr int NQ = M + 3;                                        /* quotient bits */
    const W s = XOR(a[B - 1], b[B - 1]);
    const W* ea = a + M;
    const W* eb = b + M;
    const W nzA = or_n<E>(ea), nzB = or_n<E>(eb);
    const W fA = or_n<M>(a), fB = or_n<M>(b);
    const W aspec = and_n<E>(ea), bspec = and_n<E>(eb);

    /* step 1: significands, normalised */
    W X[N1], Y[N1];
    BSFP_UNROLL
    for (int i = 0; i < M; ++i) {
        X[i] = a[i];
        Y[i] = b[i];
    }
    W tx[KT + 1], ty[KT + 1];
    if constexpr (FTZ) {
        X[M] = ~W(0u);
        Y[M] = ~W(0u);
        BSFP_UNROLL
        for (int i = 0; i <= KT; ++i) tx[i] = ty[i] = W(0u);
    } else {
        X[M] = nzA;
        Y[M] = nzB;
        W ones[KT + 1];
        BSFP_UNROLL
        for (int i = 0; i <= KT; ++i) ones[i] = ~W(0u);
        lnorm<N1, KT + 1>(X, ones, tx);
        lnorm<N1, KT + 1>(Y, ones, ty);
    }

    /* exponents: P1 = max(ea,1) + ty, P2 = max(eb,1) + tx (NU bits), then
     * D = P1 - P2 + bias - 2 + top = P1 + ~P2 + (bias - 1) + top: a carry-save
     * step of P1, ~P2 and the constant, a ripple adder with top as carry-in */
    W P1[NU], P2[NU];
    {
        W c1 = W(0u), c2 = W(0u);
        BSFP_UNROLL
        for (int i = 0; i < NU; ++i) {
            const W xa = (i == 0) ? OR(ea[0], NOT(nzA)) : (i < E ? ea[(i < E) ? i : 0] : W(0u));
            const W xb = (i == 0) ? OR(eb[0], NOT(nzB)) : (i < E ? eb[(i < E) ? i : 0] : W(0u));
            const W sy = (i <= KT) ? ty[(i <= KT) ? i : 0] : W(0u);
            const W sx = (i <= KT) ? tx[(i <= KT) ? i : 0] : W(0u);
            P1[i] = XOR3(xa, sy, c1);
            P2[i] = XOR3(xb, sx, c2);
            c1 = MAJ(xa, sy, c1);
            c2 = MAJ(xb, sx, c2);
        }
    }

    /* step 2: restoring division, Q[NQ-1] first (weight 2^(M+2)) */
    W R[M + 2], Q[NQ];
    BSFP_UNROLL
    for (int i = 0; i < N1; ++i) R[i] = X[i];
    R[M + 1] = W(0u);
    BSFP_UNROLL
    for (int j = 0; j < NQ; ++j) {
        W d[M + 2];
        W br = W(0u);
        BSFP_UNROLL
        for (int i = 0; i < M + 2; ++i) {
            const W yi = (i < N1) ? Y[(i < N1) ? i : 0] : W(0u);
            d[i] = XOR3(R[i], yi, br);
            br = MAJ(NOT(R[i]), yi, br);
        }
        const W q = NOT(br);
        Q[NQ - 1 - j] = q;
        BSFP_UNROLL
        for (int i = 0; i < M + 2; ++i) R[i] = MUX(q, d[i], R[i]);
        if (j + 1 < NQ) {
            BSFP_UNROLL
            for (int i = M + 1; i > 0; --i) R[i] = R[i - 1];
            R[0] = W(0u);
        }
    }
    const W rem = or_n<M + 2>(R);

    /* step 3: normalisation and the exponent */
    const W top = Q[NQ - 1];
    W sig[N1];
    BSFP_UNROLL
    for (int i = 0; i < N1; ++i) sig[i] = MUX(top, Q[i + 2], Q[i + 1]);
    const W g = MUX(top, Q[1], Q[0]);
    const W st = ANDOR(top, Q[0], rem);
    constexpr uint32_t KB = (uint32_t)((1 << (E - 1)) - 2) & ((1u << NU) - 1u);   /* bias - 1 */
    W D[NU];
    {
        W cs[NU], cc[NU + 1];
        cc[0] = W(0u);
        BSFP_UNROLL
        for (int i = 0; i < NU; ++i) {
            const W x1 = P1[i], x2 = NOT(P2[i]);
            const bool k = (KB >> i) & 1u;
            cs[i] = k ? NOT(XOR(x1, x2)) : XOR(x1, x2);
            cc[i + 1] = k ? OR(x1, x2) : AND(x1, x2);
        }
        W c = top;
        BSFP_UNROLL
        for (int i = 0; i < NU; ++i) {
            D[i] = XOR3(cs[i], cc[i], c);
            if (i + 1 < NU) c = MAJ(cs[i], cc[i], c);
        }
    }
    const W neg = D[NU - 1];   /* exponent field before rounding < 1 */

    /* step 4: below the normal range (gradual underflow) */
    W sigf[N1], Df[NU - 1];
    W gf = g, stf = st;
    if constexpr (FTZ) {
        BSFP_UNROLL
        for (int i = 0; i < N1; ++i) sigf[i] = sig[i];
        BSFP_UNROLL
        for (int i = 0; i < NU - 1; ++i) Df[i] = D[i];
    } else {
        constexpr int NS = M + 3;
        W q[NS];
        q[0] = OR(st, g);
        BSFP_UNROLL
        for (int p = 1; p <= M + 1; ++p) q[p] = sig[p - 1];
        q[NS - 1] = W(0u);
        W nd[NU - 1];
        BSFP_UNROLL
        for (int i = 0; i < NU - 1; ++i) nd[i] = NOT(D[i]);
        rshift_sticky<NS, NU - 1>(q, nd);
        BSFP_UNROLL
        for (int i = 0; i < N1; ++i) sigf[i] = MUX(neg, q[2 + i], sig[i]);
        gf = MUX(neg, q[1], g);
        stf = MUX(neg, q[0], st);
        BSFP_UNROLL
        for (int i = 0; i < NU - 1; ++i) Df[i] = ANDN(D[i], neg);
    }

    /* step 5: rounding, specials, encoding */
    W rup = W(0u);
    if constexpr (!RZ) rup = F3<LUT_G_AND_LS>(gf, sigf[0], stf);
    W mag[M + NU];
    assemble<M, NU - 1>(Df, sigf, rup, mag);
    const W zA = FTZ ? NOT(nzA) : NOT(OR(nzA, fA));
    const W zB = FTZ ? NOT(nzB) : NOT(OR(nzB, fB));
    const W infA = ANDN(aspec, fA), infB = ANDN(bspec, fB);
    const W nan = OR(OR(AND(aspec, fA), AND(bspec, fB)), OR(AND(infA, infB), AND(zA, zB)));
    const W spec = OR3(nan, infA, zB);
    W zero = OR(zA, infB);
    if constexpr (FTZ) zero = OR(zero, neg);
    encode<E, M, NU, RZ, W, true>(mag, spec, nan, zero, s, W(0u), r);
}

/* ---------------------------------------------------- integer vectors --- */
/* r = a + b (SUB: a - b = a + ~b + 1) modulo 2^w for w-bit unsigned (or
 * two's-complement) integers: the ripple-carry adder of Sec. 3, Fig. 2, slice
 * 0 first, one XOR3 and one MAJ per slice; the carry out of slice w-1 is
 * dropped. */
template <int w, bool SUB, class W> BSFP_HD void int_addsub(const W* a, const W* b, W* r) {
    static_assert(w >= 1 && w <= 32, "1..32-bit integers");
    /* slice 0: carry-in 0 (add) or 1 (sub) */
    W c;
    if constexpr (SUB) {
        r[0] = XOR(a[0], b[0]);          /* a0 + ~b0 + 1 */
        c = OR(a[0], NOT(b[0]));
    } else {
        r[0] = XOR(a[0], b[0]);
        c = AND(a[0], b[0]);
    }
    BSFP_UNROLL
    for (int i = 1; i < w; ++i) {
        const W bi = SUB ? NOT(b[i]) : b[i];
        r[i] = XOR3H(a[i], bi, c);
        if (i + 1 < w) c = MAJH(a[i], bi, c);
    }
}

/* r = a * b modulo 2^w: the carry-save array of the significand multiplier
 * kept to the columns below w.  Row j adds the partial products a_i b_j of
 * columns i + j < w; the carries of each row are absorbed by the next row's
 * adders in the same columns and those of the last row leave the top column,
 * so the low w sums are the product with no final adder. */
template <int w, class W> BSFP_HD void int_mul(const W* a, const W* b, W* r) {
    static_assert(w >= 1 && w <= 32, "1..32-bit integers");
    W S[w], C[w + 1];
    BSFP_UNROLL
    for (int i = 0; i < w; ++i) S[i] = AND(a[i], b[0]);
    BSFP_UNROLL
    for (int j = 1; j < w; ++j) {
        W nc[w + 1];
        BSFP_UNROLL
        for (int col = j; col < w; ++col) {
            const W pp = AND(a[col - j], b[j]);
            if (j == 1) {
                nc[col + 1] = AND(S[col], pp);
                S[col] = XOR(S[col], pp);
            } else {
                nc[col + 1] = MAJH(S[col], C[col], pp);
                S[col] = XOR3H(S[col], C[col], pp);
            }
        }
        BSFP_UNROLL
        for (int col = j + 1; col < w; ++col) C[col] = nc[col];
    }
    BSFP_UNROLL
    for (int i = 0; i < w; ++i) r[i] = S[i];
}

/* integer op codes (bsfp_int_* in bsfp.h) */
enum IntOp : int { IOP_ADD = 0, IOP_SUB = 1, IOP_MUL = 2 };

template <int w, int OP, class W> BSFP_HD void int_op(const W* a, const W* b, W* r) {
    if constexpr (OP == IOP_ADD) int_addsub<w, false>(a, b, r);
    else if constexpr (OP == IOP_SUB) int_addsub<w, true>(a, b, r);
    else int_mul<w>(a, b, r);
}

/* --------------------------------------------------------- conversions --- */
/* r (1/E/M, B slices) = x (IEEE binary32, 32 slices: slice 0 the fraction's
 * least significant bit, slice 31 the sign), rounded once in mode RZ/FTZ --
 * a narrowing conversion built as a circuit over whole words like the ops.
 * The binary32 exponent is rebiased, D = max(e,1) - 127 + bias - 1 (the
 * target's exponent field minus one), the significand keeps its M+1 top
 * bits with guard and sticky below, a target below the normal range takes
 * the right shift into the subnormal positions, and rounding, overflow and
 * the specials are those of the ops.  A binary32 subnormal is a tiny value
 * like any other (flushed under FTZ). */
template <int E, int M, bool RZ, bool FTZ = false, class W> BSFP_HD void from_f32(const W* x, W* r) {
    static_assert(E >= 2 && E <= 8 && M >= 1 && M <= 23, "narrowing from binary32 only");
    constexpr int MS = 23, ES = 8;
    constexpr int bias = (1 << (E - 1)) - 1;
    constexpr int NU = 10;                         /* D lies in [-127, 253] */
    const W s = x[31];
    const W* ex = x + MS;
    const W nz = or_n<ES>(ex);
    const W spec = and_n<ES>(ex);
    const W fx = or_n<MS>(x);
    const W nan = AND(spec, fx);

    /* D = max(e,1) + (bias - 128), NU-bit two's complement (a constant addend) */
    constexpr uint32_t K = (uint32_t)(bias - 128) & ((1u << NU) - 1u);
    W D[NU];
    {
        W c = W(0u);
        BSFP_UNROLL
        for (int i = 0; i < NU; ++i) {
            const W ai = (i == 0) ? OR(ex[0], NOT(nz)) : (i < ES ? ex[(i < ES) ? i : 0] : W(0u));
            const bool k = (K >> i) & 1u;
            D[i] = k ? NOT(XOR(ai, c)) : XOR(ai, c);
            if (i + 1 < NU) c = k ? OR(ai, c) : AND(ai, c);
        }
    }
    const W neg = D[NU - 1];

    /* the target's M+1 significand bits, guard and sticky */
    W sig[M + 1];
    BSFP_UNROLL
    for (int i = 0; i < M; ++i) sig[i] = x[MS - M + i];
    sig[M] = nz;
    const W g = (M < MS) ? x[(M < MS) ? MS - M - 1 : 0] : W(0u);
    const W st = or_n<(M < MS - 1) ? MS - M - 1 : 0>(x);

    W sigf[M + 1], Df[NU - 1];
    W gf = g, stf = st;
    if constexpr (FTZ) {
        BSFP_UNROLL
        for (int i = 0; i <= M; ++i) sigf[i] = sig[i];
        BSFP_UNROLL
        for (int i = 0; i < NU - 1; ++i) Df[i] = D[i];
    } else {
        constexpr int NQ = M + 3;
        W q[NQ];
        q[0] = OR(st, g);
        BSFP_UNROLL
        for (int p = 1; p <= M + 1; ++p) q[p] = sig[p - 1];
        q[NQ - 1] = W(0u);
        W nd[NU - 1];
        BSFP_UNROLL
        for (int i = 0; i < NU - 1; ++i) nd[i] = NOT(D[i]);
        rshift_sticky<NQ, NU - 1>(q, nd);
        BSFP_UNROLL
        for (int i = 0; i <= M; ++i) sigf[i] = MUX(neg, q[2 + i], sig[i]);
        gf = MUX(neg, q[1], g);
        stf = MUX(neg, q[0], st);
        BSFP_UNROLL
        for (int i = 0; i < NU - 1; ++i) Df[i] = ANDN(D[i], neg);
    }
    W rup = W(0u);
    if constexpr (!RZ) rup = F3<LUT_G_AND_LS>(gf, sigf[0], stf);
    W mag[M + NU];
    assemble<M, NU - 1>(Df, sigf, rup, mag);
    W zero = NOT(OR(nz, fx));
    if constexpr (FTZ) zero = OR3(zero, neg, NOT(nz));   /* tiny before rounding */
    encode<E, M, NU, RZ, W, true>(mag, spec, nan, zero, s, W(0u), r);
}

/* r (IEEE binary32, 32 slices) = x (1/E/M), exactly: every value of a format
 * with E <= 8 and M <= 23 is a binary32 value.  The significand (implicit bit
 * included) is normalised left by the log shifter as far as the binary32
 * exponent allows (subnormals of narrow-exponent formats become normal
 * binary32 values); NaN becomes the canonical binary32 NaN.  Under FTZ an
 * operand with exponent field 0 is a zero of its sign. */
template <int E, int M, bool FTZ = false, class W> BSFP_HD void to_f32(const W* x, W* r) {
    static_assert(E >= 2 && E <= 8 && M >= 1 && M <= 23, "widening to binary32 only");
    constexpr int B = 1 + E + M;
    constexpr int bias = (1 << (E - 1)) - 1;
    const W s = x[B - 1];
    const W* ex = x + M;
    const W nz = or_n<E>(ex);
    const W spec = and_n<E>(ex);
    const W fx = or_n<M>(x);
    const W nan = AND(spec, fx);

    /* um1 = max(e,1) + (127 - bias) - 1: the binary32 exponent field of 1.f,
     * minus one (8 bits; never above 253) */
    constexpr uint32_t K = (uint32_t)(126 - bias);
    W um1[8];
    {
        W c = W(0u);
        BSFP_UNROLL
        for (int i = 0; i < 8; ++i) {
            const W ai = (i == 0) ? OR(ex[0], NOT(nz)) : (i < E ? ex[(i < E) ? i : 0] : W(0u));
            const bool k = (K >> i) & 1u;
            um1[i] = k ? NOT(XOR(ai, c)) : XOR(ai, c);
            if (i + 1 < 8) c = k ? OR(ai, c) : AND(ai, c);
        }
    }
    W sig[M + 1];
    BSFP_UNROLL
    for (int i = 0; i < M; ++i) sig[i] = x[i];
    sig[M] = FTZ ? ~W(0u) : nz;
    W D[8];
    if constexpr (FTZ) {
        BSFP_UNROLL
        for (int i = 0; i < 8; ++i) D[i] = um1[i];
    } else {
        /* normalise by t = min(lz, um1), then D = um1 - t (>= 0) */
        constexpr int KT = floor_log2(M);
        W t[KT + 1];
        lnorm<M + 1, 8>(sig, um1, t);
        sub_un<8, KT + 1>(um1, t, D);
    }
    W mag8[M + 9];
    assemble<M, 8>(D, sig, W(0u), mag8);
    /* the binary32 magnitude: fraction bits M..1 at the top of the 23 */
    W mag[23 + 9];
    BSFP_UNROLL
    for (int i = 0; i < 23 + 9; ++i) mag[i] = (i < 23 - M) ? W(0u) : mag8[(i < 23 - M) ? 0 : i - (23 - M)];
    const W zero = FTZ ? NOT(nz) : NOT(OR(nz, fx));
    encode<8, 23, 9, false, W, true>(mag, spec, nan, zero, s, W(0u), r);
}

/* ----------------------------------------------------------------- ops --- */
enum Op : int { OP_ADD = 0, OP_SUB = 1, OP_MUL = 2, OP_FMA2 = 3, OP_DIV = 4 };

/* Rounding mode of a format: bit 0 = toward zero (else to nearest even),
 * bit 1 = flush to zero (operands and results below the normal range are
 * zeros of their sign). */
BSFP_HDC constexpr bool mode_rz(int R) { return (R & 1) != 0; }
BSFP_HDC constexpr bool mode_ftz(int R) { return (R & 2) != 0; }

/* r = op(a, b[, c]); fma2 = add(mul(a, b), c), each rounded; div = a / b. */
template <int E, int M, int R, int OP, class W>
BSFP_HD void fp_op(const W* a, const W* b, const W* c, W* r) {
    constexpr bool RZ = mode_rz(R), FTZ = mode_ftz(R);
    if constexpr (OP == OP_ADD) {
        fp_add<E, M, RZ, false, FTZ>(a, b, r);
    } else if constexpr (OP == OP_SUB) {
        fp_add<E, M, RZ, true, FTZ>(a, b, r);
    } else if constexpr (OP == OP_MUL) {
        fp_mul<E, M, RZ, FTZ>(a, b, r);
    } else if constexpr (OP == OP_DIV) {
        fp_div<E, M, RZ, FTZ>(a, b, r);
    } else {
        W p[1 + E + M];
        fp_mul<E, M, RZ, FTZ>(a, b, p);
        fp_add<E, M, RZ, false, FTZ>(p, c, r);
    }
}

}  // namespace bsfp
