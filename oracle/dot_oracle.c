/*
 * dot_oracle.c -- plain, slow, obviously correct CPU reference for the
 * multi-limb add / sub / mul of "Leveraging SIMD for Accelerating
 * Large-number Arithmetic" (DigitsOnTurbo).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file: only the test suite, the package's smoke check and the
 * bench's CPU-baseline leg do.  It shares no code, header, table or constant
 * with the CUDA library; it sees only the raw limb arrays.
 *
 * Number representation (Sec. 2.1, Table 2): an m-limb operand is
 * A = sum_{i<m} A_i X^i with X = 2^k; here k = 32, limbs little-endian
 * (A_0 first), one operand per row of a [batch][m] array.
 *
 * What each function computes (the plain definitions the method reaches):
 *   add : S + c_out X^m = A + B                  (Theorem 1, Sec. 3.1)
 *   sub : D - b_out X^m = A - B, b_out in {0,1}  (Sec. 3.1, "Subtraction")
 *   mul : P = A * B as exactly 2m limbs          (Theorem 2, Sec. 3.2)
 *   add_gen / sub_gen : the mpn-style variants (Sec. 3.3 and the textbook
 *         MPN-ADD-M of the appendix): S + c X^ma = A + B + cin with B of
 *         mb <= ma limbs padded with zeros (as in Theorem 2's proof), and
 *         the borrow mirror D - b X^ma = A - B - bin
 *   sqr : P = A * A as 2m limbs
 *   mul_radix : P = A * B for operands in an unsaturated radix 2^k, k <= 31
 *         (Sec. 2.1: each digit kept below 2^k inside a 32-bit word), as 2n
 *         digits each below 2^k
 * The add/sub loops are the textbook S_i = A_i + B_i + C_{i-1} recurrence
 * (Sec. 2.2 and Alg. 3, MPN-ADD-M) with 64-bit intermediates; the product is
 * the ROW-wise schoolbook (operand scanning), deliberately not the column form
 * the GPU uses.  oracle_mul_columns states the product a second way, as
 * Theorem 2's column sums followed by one carry pass, to check the column
 * identity the paper's multiplication rests on; it is not the parity target.
 *
 * Readings where the paper is silent (listed in the design notes):
 *   - limbs are 32-bit (the paper uses 64 / 52); results are radix-free;
 *   - the product has exactly 2m limbs; a carry past limb 2m-1 (Alg. 2's
 *     "prepend" case) is unreachable for A, B < X^m, so oracle_mul_columns
 *     reports it as an error;
 *   - subtraction with A < B wraps modulo X^m and returns borrow 1;
 *   - dot_add / dot_sub take no carry-in (Alg. 1 starts with c_out = 0);
 *     the variants take one, and any nonzero carry-in word counts as 1.
 *
 * All functions return 0 on success, -1 on a bad argument.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

/* ---- add: S_i = (A_i + B_i + c_i) mod X, c_{i+1} = floor(.../X) ---------- */
static void add_one(const uint32_t *a, const uint32_t *b, uint32_t *s,
                    uint32_t *carry, size_t m)
{
    uint64_t c = 0;
    for (size_t i = 0; i < m; ++i) {
        uint64_t t = (uint64_t)a[i] + (uint64_t)b[i] + c;
        s[i] = (uint32_t)t;
        c = t >> 32;
    }
    *carry = (uint32_t)c;
}

/* ---- sub: D_i = (A_i - B_i - br_i) mod X, br_{i+1} = [A_i < B_i + br_i] -- */
static void sub_one(const uint32_t *a, const uint32_t *b, uint32_t *d,
                    uint32_t *borrow, size_t m)
{
    uint64_t br = 0;
    for (size_t i = 0; i < m; ++i) {
        /* two's-complement 64-bit difference: bit 63 is set iff it went negative */
        uint64_t t = (uint64_t)a[i] - (uint64_t)b[i] - br;
        d[i] = (uint32_t)t;
        br = t >> 63;
    }
    *borrow = (uint32_t)br;
}

/* ---- mul: row-wise schoolbook into 2m limbs ------------------------------ */
static void mul_one(const uint32_t *a, const uint32_t *b, uint32_t *p, size_t m)
{
    for (size_t i = 0; i < 2 * m; ++i) p[i] = 0;
    for (size_t i = 0; i < m; ++i) {
        uint64_t c = 0;
        for (size_t j = 0; j < m; ++j) {
            /* (2^32-1)^2 + 2 (2^32-1) = 2^64 - 1: never overflows */
            uint64_t t = (uint64_t)a[i] * (uint64_t)b[j] + (uint64_t)p[i + j] + c;
            p[i + j] = (uint32_t)t;
            c = t >> 32;
        }
        p[i + m] = (uint32_t)c;
    }
}

int oracle_add(const uint32_t *a, const uint32_t *b, uint32_t *s, uint32_t *carry,
               size_t m, size_t batch)
{
    if (batch && (!carry || (m && (!a || !b || !s)))) return -1;
    for (size_t k = 0; k < batch; ++k)
        add_one(a + k * m, b + k * m, s + k * m, carry + k, m);
    return 0;
}

int oracle_sub(const uint32_t *a, const uint32_t *b, uint32_t *d, uint32_t *borrow,
               size_t m, size_t batch)
{
    if (batch && (!borrow || (m && (!a || !b || !d)))) return -1;
    for (size_t k = 0; k < batch; ++k)
        sub_one(a + k * m, b + k * m, d + k * m, borrow + k, m);
    return 0;
}

int oracle_mul(const uint32_t *a, const uint32_t *b, uint32_t *p, size_t m, size_t batch)
{
    if (batch && m && (!a || !b || !p)) return -1;
    for (size_t k = 0; k < batch; ++k)
        mul_one(a + k * m, b + k * m, p + 2 * k * m, m);
    return 0;
}

/* ---- ragged: op i has off[i+1]-off[i] limbs; products at poff[i] --------- */
int oracle_add_ragged(const uint32_t *a, const uint32_t *b, uint32_t *s, uint32_t *carry,
                      const uint64_t *off, size_t batch)
{
    if (batch && (!off || !carry)) return -1;
    for (size_t k = 0; k < batch; ++k) {
        if (off[k + 1] < off[k]) return -1;
        add_one(a + off[k], b + off[k], s + off[k], carry + k, (size_t)(off[k + 1] - off[k]));
    }
    return 0;
}

int oracle_sub_ragged(const uint32_t *a, const uint32_t *b, uint32_t *d, uint32_t *borrow,
                      const uint64_t *off, size_t batch)
{
    if (batch && (!off || !borrow)) return -1;
    for (size_t k = 0; k < batch; ++k) {
        if (off[k + 1] < off[k]) return -1;
        sub_one(a + off[k], b + off[k], d + off[k], borrow + k, (size_t)(off[k + 1] - off[k]));
    }
    return 0;
}

int oracle_mul_ragged(const uint32_t *a, const uint32_t *b, uint32_t *p,
                      const uint64_t *off, const uint64_t *poff, size_t batch)
{
    if (batch && (!off || !poff)) return -1;
    for (size_t k = 0; k < batch; ++k) {
        if (off[k + 1] < off[k]) return -1;
        mul_one(a + off[k], b + off[k], p + poff[k], (size_t)(off[k + 1] - off[k]));
    }
    return 0;
}

/* ---- mixed ragged: op[i] in {0 add, 1 sub, 2 mul}; carry[i] = carry/borrow
 *      of an add/sub, 0 for a product ---------------------------------------- */
int oracle_mixed(const uint32_t *op, const uint32_t *mlimbs, const uint64_t *a_off,
                 const uint64_t *b_off, const uint64_t *r_off, size_t nops,
                 const uint32_t *a, const uint32_t *b, uint32_t *r, uint32_t *carry)
{
    if (nops && (!op || !mlimbs || !a_off || !b_off || !r_off || !carry)) return -1;
    for (size_t i = 0; i < nops; ++i) {
        size_t m = mlimbs[i];
        switch (op[i]) {
        case 0: add_one(a + a_off[i], b + b_off[i], r + r_off[i], carry + i, m); break;
        case 1: sub_one(a + a_off[i], b + b_off[i], r + r_off[i], carry + i, m); break;
        case 2: mul_one(a + a_off[i], b + b_off[i], r + r_off[i], m); carry[i] = 0; break;
        default: return -1;
        }
    }
    return 0;
}

/* ---- Theorem 2's column form: A * B = sum_c S_c X^c ----------------------
 * S_c = sum over the index pairs (i, j) with i + j = c of A_i B_j, for the
 * 2m - 1 columns c = 0 .. 2m-2.  A column sum exceeds one limb, so it is kept
 * as two 64-bit words: `lo` sums the low 32-bit halves of its products and
 * `hi` their high halves, S_c = lo + hi X (each word below m 2^32).  The
 * product's limbs then come out of one pass from the least significant end,
 * limb c taking column c's `lo`, column c-1's `hi` and the running carry.
 * This is the paper's identity with none of the SIMD staging (no gathered
 * operand arrays, no stored half products); it is a second, independent
 * statement of the product next to the row-wise schoolbook above.  A carry
 * left over after limb 2m-1 would mean a (2m+1)-limb product, impossible for
 * m-limb operands: it is reported as -2. */
static int columns_one(const uint32_t *A, const uint32_t *B, uint32_t *P, size_t m,
                       uint64_t *lo, uint64_t *hi)
{
    for (size_t c = 0; c + 1 < 2 * m; ++c) {
        const size_t i_first = c >= m ? c - (m - 1) : 0;
        const size_t i_last = c < m ? c : m - 1;
        uint64_t l = 0, h = 0;
        for (size_t i = i_first; i <= i_last; ++i) {
            const uint64_t prod = (uint64_t)A[i] * (uint64_t)B[c - i];
            l += prod & 0xFFFFFFFFu;
            h += prod >> 32;
        }
        lo[c] = l;
        hi[c] = h;
    }
    uint64_t carry = 0;
    for (size_t c = 0; c < 2 * m; ++c) {
        uint64_t t = carry;
        if (c + 1 < 2 * m) t += lo[c];
        if (c >= 1) t += hi[c - 1];
        P[c] = (uint32_t)t;
        carry = t >> 32;
    }
    return carry ? -2 : 0;
}

int oracle_mul_columns(const uint32_t *a, const uint32_t *b, uint32_t *p, size_t m, size_t batch)
{
    if (batch && m && (!a || !b || !p)) return -1;
    if (!m || !batch) return 0;
    uint64_t *lo = malloc(2 * m * sizeof *lo), *hi = malloc(2 * m * sizeof *hi);
    int rc = (lo && hi) ? 0 : -4;
    for (size_t k = 0; k < batch && rc == 0; ++k)
        rc = columns_one(a + k * m, b + k * m, p + 2 * k * m, m, lo, hi);
    free(lo);
    free(hi);
    return rc;
}

/* The index pairs of each column, column by column (c = 0 .. 2m-2) and, inside
 * a column, by ascending i: the order in which Sec. 3.2's m = 5 walkthrough
 * lists them.  ia, jb hold m*m entries; ncol holds the 2m-1 pair counts. */
int oracle_column_pairs(size_t m, int32_t *ia, int32_t *jb, int32_t *ncol)
{
    if (!m || !ia || !jb || !ncol) return -1;
    size_t t = 0;
    for (size_t c = 0; c + 1 < 2 * m; ++c) {
        const size_t i_first = c >= m ? c - (m - 1) : 0;
        const size_t i_last = c < m ? c : m - 1;
        for (size_t i = i_first; i <= i_last; ++i, ++t) {
            ia[t] = (int32_t)i;
            jb[t] = (int32_t)(c - i);
        }
        ncol[c] = (int32_t)(i_last - i_first + 1);
    }
    return t == m * m ? 0 : -3;
}

/* ---- mpn-style variants: B zero-padded to ma limbs, carry/borrow-in ------ */
static void add_gen_one(const uint32_t *a, size_t ma, const uint32_t *b, size_t mb,
                        uint32_t cin, uint32_t *s, uint32_t *carry)
{
    uint64_t c = cin ? 1u : 0u;
    for (size_t i = 0; i < ma; ++i) {
        const uint64_t bi = i < mb ? (uint64_t)b[i] : 0u;
        const uint64_t t = (uint64_t)a[i] + bi + c;
        s[i] = (uint32_t)t;
        c = t >> 32;
    }
    *carry = (uint32_t)c;
}

static void sub_gen_one(const uint32_t *a, size_t ma, const uint32_t *b, size_t mb,
                        uint32_t bin, uint32_t *d, uint32_t *borrow)
{
    uint64_t br = bin ? 1u : 0u;
    for (size_t i = 0; i < ma; ++i) {
        const uint64_t bi = i < mb ? (uint64_t)b[i] : 0u;
        const uint64_t t = (uint64_t)a[i] - bi - br;   /* bit 63 set iff negative */
        d[i] = (uint32_t)t;
        br = t >> 63;
    }
    *borrow = (uint32_t)br;
}

/* a: [batch][ma], b: [batch][mb] (mb <= ma), cin: [batch] or NULL (no
 * carry-in), s: [batch][ma], carry: [batch] */
int oracle_add_gen(const uint32_t *a, size_t ma, const uint32_t *b, size_t mb, const uint32_t *cin,
                   uint32_t *s, uint32_t *carry, size_t batch)
{
    if (mb > ma) return -1;
    if (batch && (!carry || (ma && (!a || !s)) || (mb && !b))) return -1;
    for (size_t k = 0; k < batch; ++k)
        add_gen_one(a + k * ma, ma, b + k * mb, mb, cin ? cin[k] : 0u, s + k * ma, carry + k);
    return 0;
}

int oracle_sub_gen(const uint32_t *a, size_t ma, const uint32_t *b, size_t mb, const uint32_t *bin,
                   uint32_t *d, uint32_t *borrow, size_t batch)
{
    if (mb > ma) return -1;
    if (batch && (!borrow || (ma && (!a || !d)) || (mb && !b))) return -1;
    for (size_t k = 0; k < batch; ++k)
        sub_gen_one(a + k * ma, ma, b + k * mb, mb, bin ? bin[k] : 0u, d + k * ma, borrow + k);
    return 0;
}

/* P = A * A: the definition, through the same row-wise schoolbook */
int oracle_sqr(const uint32_t *a, uint32_t *p, size_t m, size_t batch)
{
    if (batch && m && (!a || !p)) return -1;
    for (size_t k = 0; k < batch; ++k)
        mul_one(a + k * m, a + k * m, p + 2 * k * m, m);
    return 0;
}

/* ---- unsaturated radix: n digits of k bits (k <= 31), each in a 32-bit word.
 * P = A * B as exactly 2n digits below 2^k, by the row-wise schoolbook in radix
 * 2^k: t = a_i b_j + p_{i+j} + c < 2^(2k) + 2^(k+1) fits 64 bits.  Returns -1
 * on a bad argument or an input digit of 2^k or more. */
int oracle_mul_radix(const uint32_t *a, const uint32_t *b, uint32_t *p, size_t n, size_t batch,
                     unsigned k)
{
    if (k < 1 || k > 31) return -1;
    if (batch && n && (!a || !b || !p)) return -1;
    const uint64_t mask = ((uint64_t)1 << k) - 1;
    for (size_t r = 0; r < batch; ++r) {
        const uint32_t *x = a + r * n, *y = b + r * n;
        uint32_t *z = p + 2 * r * n;
        for (size_t i = 0; i < n; ++i)
            if (x[i] > mask || y[i] > mask) return -1;
        for (size_t i = 0; i < 2 * n; ++i) z[i] = 0;
        for (size_t i = 0; i < n; ++i) {
            uint64_t c = 0;
            for (size_t j = 0; j < n; ++j) {
                const uint64_t t = (uint64_t)x[i] * (uint64_t)y[j] + (uint64_t)z[i + j] + c;
                z[i + j] = (uint32_t)(t & mask);
                c = t >> k;
            }
            z[i + n] = (uint32_t)c;
        }
    }
    return 0;
}
