/*
 * symphase_oracle.c -- plain, slow CPU oracle of the symbolic-phase tableau
 * algorithm (arXiv 2311.03906).  TEST INFRASTRUCTURE ONLY: the tests, the
 * smoke check and the benchmark's CPU-baseline leg call it; the CUDA library
 * never does, and the two share no code.
 *
 * What it computes, step by step, in the paper's order:
 *   Sec. 2 (Eq. stabilizer1)  A-G tableau with destabilizers, rows 0..n-1
 *                             destabilizers, rows n..2n-1 stabilizers.
 *   Sec. 3.2.1               every phase is a bit-vector over symbols
 *                             s_0..s_ns, s_0 = the constant 1.
 *   Sec. 3.2.2 (Eq. stabilizer3, Init-C / Init-P / Init-M)
 *                             Clifford gates update x, z and phase column 0;
 *                             a fault X^{s_j} (Z^{s_j}) updates column j like
 *                             an X (Z) gate (Fact 1); a measurement follows
 *                             A-G, every rowsum also XORs symbol columns.
 *   Sec. 3.2.3 (Eq. sampling)  one shot = parity(m_k . b) with b_0 = 1.
 *
 * Readings where the paper is silent or inconsistent (each also listed in
 * the design notes):
 *   - random outcome: the new stabilizer row p gets phase e_s (only row p),
 *     which reproduces the printed tableaux of the Sec. 3.1 two-qubit example;
 *   - R / MR: measure, then the conditional Pauli X^e (e = the outcome's
 *     expression) on the measured qubit (the conditional-Pauli idea of the
 *     conclusion), applied to every row like Fact 1 does;
 *   - feed-forward X_IF / Y_IF / Z_IF (k, q): the Pauli on qubit q applied
 *     when record rec[-k] is 1, i.e. the conditional Pauli P^e with e that
 *     record's expression (Sec. 6): every row anticommuting with P gets e
 *     added to its phase;
 *   - symbols are numbered in op order: a fault's symbols when it is reached
 *     (X/Y/Z_ERROR 1, DEPOLARIZE1 2 = x,z, DEPOLARIZE2 4 = x_a,z_a,x_b,z_b),
 *     a random measurement's symbol at that measurement;
 *   - draws: Philox4x32-10 (Salmon et al., SC'11) with key (seed lo, seed
 *     hi), counter (shot lo, shot hi, channel/4, 0), word channel%4;
 *     Bernoulli u < T with T = floor(p 2^32) (p = 1 -> 2^32-1); a random
 *     measurement is a channel with T = 2^31; DEPOLARIZE1/2 draw
 *     k = floor(u*m/T) (m = 3 / 15) when u < T, and symbol s0+i takes bit i
 *     of k+1;
 *   - detector and observable rows are XORs of measurement rows; a row with
 *     a random-measurement symbol is rejected.
 * Expectations (FP64): E_j = (-1)^{c_j} prod_c (1 - 2 P_c(odd)), with
 * P_c(odd) found by enumerating the channel's outcomes.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
    OR_H = 0, OR_S, OR_CX, OR_X, OR_Y, OR_Z, OR_M, OR_MR, OR_R,
    OR_XERR, OR_YERR, OR_ZERR, OR_DEP1, OR_DEP2, OR_DET, OR_OBS, OR_TICK,
    OR_XIF, OR_YIF, OR_ZIF   /* feed-forward: targets are (look-back k, qubit) pairs */
};
enum { CH_XERR = 0, CH_YERR, CH_ZERR, CH_DEP1, CH_DEP2, CH_RANDOM };
enum {
    OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_OP = 2, OR_ERR_NONDET = 3, OR_ERR_MEM = 4
};

typedef struct {
    int64_t n;          /* qubits */
    int64_t cap;        /* symbol capacity (excluding s_0) */
    int64_t pw;         /* 64-bit words per phase row: ceil((cap+1)/64) */
    uint8_t *x, *z;     /* [(2n+1) * n] bytes; row 2n is the A-G scratch row */
    uint64_t *ph;       /* [(2n+1) * pw] phase bit-vectors */
    int64_t ns;         /* symbols allocated so far */
    int64_t nch;        /* channels allocated so far */
    int32_t *ch_type;
    double *ch_p;
    uint32_t *ch_T;
    int64_t *ch_sym0;
    int32_t *ch_nsym;
    uint8_t *sym_random; /* [cap+1] 1 if the symbol is a random-measurement one */
    int64_t nmeas, ndet, nobs;
    uint64_t *meas, *det, *obs; /* rows of pw words */
    int32_t status;
    int64_t bad_row;    /* detector (or -1-observable) index on NONDET */
} orc_prog;

/* ------------------------------------------------------------------ bits */
static inline int getb(const uint64_t *v, int64_t k) { return (int)((v[k >> 6] >> (k & 63)) & 1u); }
static inline void flipb(uint64_t *v, int64_t k) { v[k >> 6] ^= (uint64_t)1 << (k & 63); }
static inline uint8_t *X(orc_prog *P, int64_t r) { return P->x + r * P->n; }
static inline uint8_t *Z(orc_prog *P, int64_t r) { return P->z + r * P->n; }
static inline uint64_t *PH(orc_prog *P, int64_t r) { return P->ph + r * P->pw; }

/* ---------------------------------------------------------------- Philox */
/* Philox4x32-10 from its published definition: per round,
 *   (hi0,lo0) = M0*c0, (hi1,lo1) = M1*c2,
 *   c = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0),
 * and the key is bumped by the Weyl constants between rounds. */
void or_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

uint32_t or_threshold(double p)
{
    if (!(p > 0.0)) return 0u;
    double t = floor(p * 4294967296.0);
    if (t >= 4294967295.0) return 4294967295u;
    return (uint32_t)t;
}

/* the 32-bit uniform word of channel c in shot `shot` */
static uint32_t channel_word(uint64_t seed, uint64_t shot, int64_t c)
{
    uint32_t ctr[4] = {(uint32_t)shot, (uint32_t)(shot >> 32), (uint32_t)(c / 4), 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    or_philox(ctr, key, out);
    return out[c % 4];
}

/* outcome index of a channel: 0 = nothing happened, else the symbol bits
 * as an integer whose bit i is symbol s0+i */
static uint32_t channel_outcome(int32_t type, uint32_t T, uint32_t u)
{
    if (u >= T) return 0u;
    if (type == CH_DEP1) return (uint32_t)(((uint64_t)u * 3u) / T) + 1u;
    if (type == CH_DEP2) return (uint32_t)(((uint64_t)u * 15u) / T) + 1u;
    return 1u;
}

/* ------------------------------------------------------------- tableau */
/* A-G's g: the power of i picked up when the single-qubit Paulis (x1,z1)
 * and (x2,z2) are multiplied in that order. */
static int g_func(int x1, int z1, int x2, int z2)
{
    if (!x1 && !z1) return 0;
    if (x1 && z1) return z2 - x2;
    if (x1 && !z1) return z2 * (2 * x2 - 1);
    return x2 * (1 - 2 * z2);
}

/* rowsum(h, i): row h := P_i * P_h.  Column 0 of the phase takes A-G's
 * g-sum; columns 1..ns are XORed (Init-M). */
static void rowsum(orc_prog *P, int64_t h, int64_t i)
{
    int64_t n = P->n;
    uint8_t *xh = X(P, h), *zh = Z(P, h), *xi = X(P, i), *zi = Z(P, i);
    uint64_t *ph = PH(P, h), *pi = PH(P, i);
    int64_t tot = 2 * getb(ph, 0) + 2 * getb(pi, 0);
    for (int64_t j = 0; j < n; j++) tot += g_func(xi[j], zi[j], xh[j], zh[j]);
    tot = ((tot % 4) + 4) % 4;
    int r0 = (tot >= 2) ? 1 : 0; /* 0 or 2 for commuting rows */
    for (int64_t w = 0; w < P->pw; w++) ph[w] ^= pi[w];
    /* column 0 is set from the g-sum rather than XORed */
    if (getb(ph, 0) != r0) flipb(ph, 0);
    for (int64_t j = 0; j < n; j++) { xh[j] ^= xi[j]; zh[j] ^= zi[j]; }
}

static void gate_h(orc_prog *P, int64_t a)
{
    for (int64_t r = 0; r < 2 * P->n; r++) {
        uint8_t *x = X(P, r), *z = Z(P, r);
        if (x[a] & z[a]) flipb(PH(P, r), 0);
        uint8_t t = x[a]; x[a] = z[a]; z[a] = t;
    }
}

static void gate_s(orc_prog *P, int64_t a)
{
    for (int64_t r = 0; r < 2 * P->n; r++) {
        uint8_t *x = X(P, r), *z = Z(P, r);
        if (x[a] & z[a]) flipb(PH(P, r), 0);
        z[a] ^= x[a];
    }
}

static void gate_cx(orc_prog *P, int64_t a, int64_t b)
{
    for (int64_t r = 0; r < 2 * P->n; r++) {
        uint8_t *x = X(P, r), *z = Z(P, r);
        if (x[a] & z[b] & (x[b] ^ z[a] ^ 1)) flipb(PH(P, r), 0);
        x[b] ^= x[a];
        z[a] ^= z[b];
    }
}

/* Fact 1 with an exponent: column `col` of every row flips where the Pauli
 * (px, pz) anticommutes with the row's Pauli on qubit a. */
static void pauli_column(orc_prog *P, int64_t a, int px, int pz, int64_t col)
{
    for (int64_t r = 0; r < 2 * P->n; r++) {
        int flip = (px & Z(P, r)[a]) ^ (pz & X(P, r)[a]);
        if (flip) flipb(PH(P, r), col);
    }
}

static int64_t new_symbol(orc_prog *P, int random)
{
    P->ns += 1;
    P->sym_random[P->ns] = (uint8_t)random;
    return P->ns;
}

static void new_channel(orc_prog *P, int32_t type, double p, int64_t sym0, int32_t nsym)
{
    int64_t c = P->nch++;
    P->ch_type[c] = type;
    P->ch_p[c] = p;
    P->ch_T[c] = (type == CH_RANDOM) ? 0x80000000u : or_threshold(p);
    P->ch_sym0[c] = sym0;
    P->ch_nsym[c] = nsym;
}

/* Init-M on qubit a; the outcome's bit-vector is left in `out` (pw words). */
static void measure(orc_prog *P, int64_t a, uint64_t *out)
{
    int64_t n = P->n;
    int64_t p = -1;
    for (int64_t i = n; i < 2 * n; i++) if (X(P, i)[a]) { p = i; break; }
    if (p >= 0) {
        /* random outcome */
        for (int64_t i = 0; i < 2 * n; i++)
            if (i != p && X(P, i)[a]) rowsum(P, i, p);
        memcpy(X(P, p - n), X(P, p), (size_t)n);
        memcpy(Z(P, p - n), Z(P, p), (size_t)n);
        memcpy(PH(P, p - n), PH(P, p), (size_t)P->pw * 8);
        memset(X(P, p), 0, (size_t)n);
        memset(Z(P, p), 0, (size_t)n);
        Z(P, p)[a] = 1;
        int64_t s = new_symbol(P, 1);
        new_channel(P, CH_RANDOM, 0.5, s, 1);
        memset(PH(P, p), 0, (size_t)P->pw * 8);
        flipb(PH(P, p), s);
        memcpy(out, PH(P, p), (size_t)P->pw * 8);
    } else {
        /* deterministic outcome: accumulate in the scratch row 2n */
        int64_t sc = 2 * n;
        memset(X(P, sc), 0, (size_t)n);
        memset(Z(P, sc), 0, (size_t)n);
        memset(PH(P, sc), 0, (size_t)P->pw * 8);
        for (int64_t i = 0; i < n; i++)
            if (X(P, i)[a]) rowsum(P, sc, i + n);
        memcpy(out, PH(P, sc), (size_t)P->pw * 8);
    }
}

/* The Pauli X^xb Z^zb on qubit a applied when the affine form e is 1
 * (Sec. 6, conditional Paulis): every row that anticommutes with it, i.e.
 * with xb*z_a + zb*x_a odd, gets e added to its phase.  A reset is the
 * conditional X^e with e the outcome just measured. */
static void cond_pauli(orc_prog *P, int64_t a, int xb, int zb, const uint64_t *e)
{
    for (int64_t r = 0; r < 2 * P->n; r++) {
        if ((xb && Z(P, r)[a]) ^ (zb && X(P, r)[a])) {
            uint64_t *ph = PH(P, r);
            for (int64_t w = 0; w < P->pw; w++) ph[w] ^= e[w];
        }
    }
}

void or_free(orc_prog *P)
{
    if (!P) return;
    free(P->x); free(P->z); free(P->ph);
    free(P->ch_type); free(P->ch_p); free(P->ch_T); free(P->ch_sym0); free(P->ch_nsym);
    free(P->sym_random); free(P->meas); free(P->det); free(P->obs);
    free(P);
}

/*
 * Build the program of a circuit: ops i = 0..nops-1 with code[i], targets
 * tg[off[i] .. off[i+1]) and argument arg[i].  `stop` (< nops) stops after
 * that many ops, for inspecting intermediate tableaux.  Returns NULL only on
 * allocation failure; otherwise check ->status.
 */
orc_prog *or_build(int64_t nq, int64_t nops, const int32_t *code, const int64_t *off,
                   const int32_t *tg, const double *arg, int64_t stop)
{
    orc_prog *P = (orc_prog *)calloc(1, sizeof(orc_prog));
    if (!P) return NULL;
    if (stop < 0 || stop > nops) stop = nops;
    P->n = nq;
    /* capacity: every fault symbol plus one per measurement or reset */
    int64_t cap = 0, nmeas = 0, ndet = 0, nobs = 0;
    for (int64_t i = 0; i < nops; i++) {
        int64_t k = off[i + 1] - off[i];
        switch (code[i]) {
        case OR_XERR: case OR_YERR: case OR_ZERR: cap += k; break;
        case OR_DEP1: cap += 2 * k; break;
        case OR_DEP2: cap += 2 * k; break;
        case OR_M: case OR_MR: cap += k; nmeas += k; break;
        case OR_R: cap += k; break;
        case OR_DET: ndet++; break;
        case OR_OBS: if ((int64_t)arg[i] + 1 > nobs) nobs = (int64_t)arg[i] + 1; break;
        default: break;
        }
    }
    P->cap = cap;
    P->pw = (cap + 1 + 63) / 64;
    int64_t rows = 2 * nq + 1;
    P->x = (uint8_t *)calloc((size_t)(rows * nq + 1), 1);
    P->z = (uint8_t *)calloc((size_t)(rows * nq + 1), 1);
    P->ph = (uint64_t *)calloc((size_t)(rows * P->pw), 8);
    P->ch_type = (int32_t *)calloc((size_t)cap + 1, 4);
    P->ch_p = (double *)calloc((size_t)cap + 1, 8);
    P->ch_T = (uint32_t *)calloc((size_t)cap + 1, 4);
    P->ch_sym0 = (int64_t *)calloc((size_t)cap + 1, 8);
    P->ch_nsym = (int32_t *)calloc((size_t)cap + 1, 4);
    P->sym_random = (uint8_t *)calloc((size_t)cap + 2, 1);
    P->meas = (uint64_t *)calloc((size_t)(nmeas + 1) * P->pw, 8);
    P->det = (uint64_t *)calloc((size_t)(ndet + 1) * P->pw, 8);
    P->obs = (uint64_t *)calloc((size_t)(nobs + 1) * P->pw, 8);
    uint64_t *e = (uint64_t *)calloc((size_t)P->pw, 8);
    if (!P->x || !P->z || !P->ph || !P->ch_type || !P->ch_p || !P->ch_T || !P->ch_sym0 ||
        !P->ch_nsym || !P->sym_random || !P->meas || !P->det || !P->obs || !e) {
        free(e); or_free(P); return NULL;
    }
    /* initial state |0...0>: destabilizer i = X_i, stabilizer i = Z_i */
    for (int64_t i = 0; i < nq; i++) { X(P, i)[i] = 1; Z(P, nq + i)[i] = 1; }
    P->bad_row = 0;

    for (int64_t i = 0; i < stop && P->status == OR_OK; i++) {
        const int32_t *t = tg + off[i];
        int64_t k = off[i + 1] - off[i];
        int c = code[i];
        for (int64_t j = 0; j < k; j++) {
            if (c == OR_DET || c == OR_OBS || c == OR_TICK) break;
            if ((c == OR_XIF || c == OR_YIF || c == OR_ZIF) && !(j & 1)) continue;   /* look-backs */
            if (t[j] < 0 || t[j] >= nq) { P->status = OR_ERR_ARG; break; }
        }
        if (P->status) break;
        if ((c == OR_CX || c == OR_DEP2 || c == OR_XIF || c == OR_YIF || c == OR_ZIF) && (k % 2)) {
            P->status = OR_ERR_ARG;
            break;
        }
        if (c >= OR_XERR && c <= OR_DEP2 && !(arg[i] >= 0.0 && arg[i] <= 1.0)) { P->status = OR_ERR_ARG; break; }
        switch (c) {
        case OR_H: for (int64_t j = 0; j < k; j++) gate_h(P, t[j]); break;
        case OR_S: for (int64_t j = 0; j < k; j++) gate_s(P, t[j]); break;
        case OR_CX:
            for (int64_t j = 0; j < k; j += 2) {
                if (t[j] == t[j + 1]) { P->status = OR_ERR_ARG; break; }
                gate_cx(P, t[j], t[j + 1]);
            }
            break;
        case OR_X: for (int64_t j = 0; j < k; j++) pauli_column(P, t[j], 1, 0, 0); break;
        case OR_Y: for (int64_t j = 0; j < k; j++) pauli_column(P, t[j], 1, 1, 0); break;
        case OR_Z: for (int64_t j = 0; j < k; j++) pauli_column(P, t[j], 0, 1, 0); break;
        case OR_XERR: case OR_YERR: case OR_ZERR:
            for (int64_t j = 0; j < k; j++) {
                int64_t s = new_symbol(P, 0);
                new_channel(P, c == OR_XERR ? CH_XERR : (c == OR_YERR ? CH_YERR : CH_ZERR), arg[i], s, 1);
                pauli_column(P, t[j], c != OR_ZERR, c != OR_XERR, s);
            }
            break;
        case OR_DEP1:
            for (int64_t j = 0; j < k; j++) {
                int64_t s = new_symbol(P, 0);
                new_symbol(P, 0);
                new_channel(P, CH_DEP1, arg[i], s, 2);
                pauli_column(P, t[j], 1, 0, s);     /* X^{s}   */
                pauli_column(P, t[j], 0, 1, s + 1); /* Z^{s+1} */
            }
            break;
        case OR_DEP2:
            for (int64_t j = 0; j < k; j += 2) {
                if (t[j] == t[j + 1]) { P->status = OR_ERR_ARG; break; }
                int64_t s = new_symbol(P, 0);
                new_symbol(P, 0); new_symbol(P, 0); new_symbol(P, 0);
                new_channel(P, CH_DEP2, arg[i], s, 4);
                pauli_column(P, t[j], 1, 0, s);
                pauli_column(P, t[j], 0, 1, s + 1);
                pauli_column(P, t[j + 1], 1, 0, s + 2);
                pauli_column(P, t[j + 1], 0, 1, s + 3);
            }
            break;
        case OR_M: case OR_MR: case OR_R:
            for (int64_t j = 0; j < k; j++) {
                measure(P, t[j], e);
                if (c != OR_R) {
                    memcpy(P->meas + P->nmeas * P->pw, e, (size_t)P->pw * 8);
                    P->nmeas++;
                }
                if (c != OR_M) cond_pauli(P, t[j], 1, 0, e);
            }
            break;
        case OR_DET: case OR_OBS: {
            uint64_t *row;
            if (c == OR_DET) row = P->det + (P->ndet++) * P->pw;
            else {
                int64_t o = (int64_t)arg[i];
                if (o < 0) { P->status = OR_ERR_ARG; break; }
                row = P->obs + o * P->pw;
                if (o + 1 > P->nobs) P->nobs = o + 1;
            }
            for (int64_t j = 0; j < k; j++) {
                int64_t lb = t[j];
                if (lb < 1 || lb > P->nmeas) { P->status = OR_ERR_ARG; break; }
                const uint64_t *m = P->meas + (P->nmeas - lb) * P->pw;
                for (int64_t w = 0; w < P->pw; w++) row[w] ^= m[w];
            }
            break;
        }
        case OR_XIF: case OR_YIF: case OR_ZIF:
            for (int64_t j = 0; j < k; j += 2) {
                int64_t lb = t[j];
                if (lb < 1 || lb > P->nmeas) { P->status = OR_ERR_ARG; break; }
                cond_pauli(P, t[j + 1], c != OR_ZIF, c != OR_XIF, P->meas + (P->nmeas - lb) * P->pw);
            }
            break;
        case OR_TICK: break;
        default: P->status = OR_ERR_OP; break;
        }
    }
    free(e);
    if (P->status != OR_OK) return P;
    /* a detector or observable that depends on a random-measurement symbol
     * is not deterministic */
    for (int64_t d = 0; d < P->ndet + P->nobs && P->status == OR_OK; d++) {
        const uint64_t *row = d < P->ndet ? P->det + d * P->pw : P->obs + (d - P->ndet) * P->pw;
        for (int64_t s = 1; s <= P->ns; s++)
            if (P->sym_random[s] && getb(row, s)) {
                P->status = OR_ERR_NONDET;
                P->bad_row = d < P->ndet ? d : -1 - (d - P->ndet);
                break;
            }
    }
    return P;
}

/* out: status, n, nmeas, ndet, nobs, ns, nch, pw, bad_row */
void or_info(const orc_prog *P, int64_t *out)
{
    out[0] = P->status; out[1] = P->n; out[2] = P->nmeas; out[3] = P->ndet;
    out[4] = P->nobs; out[5] = P->ns; out[6] = P->nch; out[7] = P->pw; out[8] = P->bad_row;
}

/* which: 0 meas, 1 det, 2 obs; rows copied as pw words each */
void or_rows(const orc_prog *P, int32_t which, uint64_t *out)
{
    const uint64_t *src = which == 0 ? P->meas : (which == 1 ? P->det : P->obs);
    int64_t cnt = which == 0 ? P->nmeas : (which == 1 ? P->ndet : P->nobs);
    memcpy(out, src, (size_t)(cnt * P->pw) * 8);
}

void or_channels(const orc_prog *P, int32_t *type, double *p, uint32_t *T, int64_t *sym0, int32_t *nsym)
{
    for (int64_t c = 0; c < P->nch; c++) {
        type[c] = P->ch_type[c]; p[c] = P->ch_p[c]; T[c] = P->ch_T[c];
        sym0[c] = P->ch_sym0[c]; nsym[c] = P->ch_nsym[c];
    }
}

void or_random_symbols(const orc_prog *P, uint8_t *flag)
{
    memcpy(flag, P->sym_random, (size_t)P->ns + 1);
}

/* The full tableau after build (rows 0..2n-1): x, z as bytes, phases. */
void or_tableau(orc_prog *P, uint8_t *x, uint8_t *z, uint64_t *ph)
{
    memcpy(x, P->x, (size_t)(2 * P->n * P->n));
    memcpy(z, P->z, (size_t)(2 * P->n * P->n));
    memcpy(ph, P->ph, (size_t)(2 * P->n * P->pw) * 8);
}

/* b for one shot: bit 0 = 1 (s_0), bit s = drawn value of symbol s */
void or_draw(const orc_prog *P, uint64_t seed, uint64_t shot, uint64_t *b)
{
    memset(b, 0, (size_t)P->pw * 8);
    b[0] = 1u;
    for (int64_t c = 0; c < P->nch; c++) {
        uint32_t u = channel_word(seed, shot, c);
        uint32_t v = channel_outcome(P->ch_type[c], P->ch_T[c], u);
        for (int32_t i = 0; i < P->ch_nsym[c]; i++)
            if ((v >> i) & 1u) flipb(b, P->ch_sym0[c] + i);
    }
}

static int parity_dot(const uint64_t *a, const uint64_t *b, int64_t pw)
{
    uint64_t acc = 0;
    for (int64_t w = 0; w < pw; w++) acc ^= a[w] & b[w];
    return __builtin_parityll(acc);
}

/* records of one shot for a given b; outputs are packed little-endian bits */
void or_eval(const orc_prog *P, const uint64_t *b, uint64_t *meas, uint64_t *det, uint64_t *obs)
{
    int64_t wm = (P->nmeas + 63) / 64, wd = (P->ndet + 63) / 64, wo = (P->nobs + 63) / 64;
    memset(meas, 0, (size_t)wm * 8);
    memset(det, 0, (size_t)wd * 8);
    memset(obs, 0, (size_t)wo * 8);
    for (int64_t j = 0; j < P->nmeas; j++)
        if (parity_dot(P->meas + j * P->pw, b, P->pw)) flipb(meas, j);
    for (int64_t j = 0; j < P->ndet; j++)
        if (parity_dot(P->det + j * P->pw, b, P->pw)) flipb(det, j);
    for (int64_t j = 0; j < P->nobs; j++)
        if (parity_dot(P->obs + j * P->pw, b, P->pw)) flipb(obs, j);
}

/* records of the listed shots (global shot indices), shot-major */
void or_sample_shots(const orc_prog *P, uint64_t seed, const uint64_t *shots, int64_t nshots,
                     uint64_t *meas, uint64_t *det, uint64_t *obs)
{
    int64_t wm = (P->nmeas + 63) / 64, wd = (P->ndet + 63) / 64, wo = (P->nobs + 63) / 64;
    uint64_t *b = (uint64_t *)malloc((size_t)P->pw * 8);
    if (!b) return;
    for (int64_t t = 0; t < nshots; t++) {
        or_draw(P, seed, shots[t], b);
        or_eval(P, b, meas + t * wm, det + t * wd, obs + t * wo);
    }
    free(b);
}

void or_sample(const orc_prog *P, uint64_t seed, uint64_t shot0, int64_t nshots,
               uint64_t *meas, uint64_t *det, uint64_t *obs)
{
    int64_t wm = (P->nmeas + 63) / 64, wd = (P->ndet + 63) / 64, wo = (P->nobs + 63) / 64;
    uint64_t *b = (uint64_t *)malloc((size_t)P->pw * 8);
    if (!b) return;
    for (int64_t t = 0; t < nshots; t++) {
        or_draw(P, seed, shot0 + (uint64_t)t, b);
        or_eval(P, b, meas + t * wm, det + t * wd, obs + t * wo);
    }
    free(b);
}

/* ------------------------------------------------ grouped draw (stream 2) */
/* An opt-in second definition of "sample b from P_C" (Algorithm 1), exact
 * for the same Sec. 3.1 distributions but drawing far fewer words when the
 * channels rarely fire.  Counter word 3 tells the streams apart (the first
 * stream uses 0):
 *   - random-measurement channel of rank r (in channel order): bit r%32 of
 *     word (r/32)%4 of Philox(counter (shot lo, shot hi, r/128, 3));
 *   - the other channels, in channel order, form groups of 32; group g
 *     fires with probability 1 - prod_i (1 - p_i): word g%4 of Philox(
 *     counter (shot lo, shot hi, g/4, 1)) below G_g = floor((1 - prod) 2^32);
 *   - in a group that fired, channel i (word i%4 of Philox(counter (shot lo,
 *     shot hi, 8g + i/4, 2))) is the first to fire with probability
 *     q_i = p_i / (1 - R_i), R_i = prod_{j >= i} (1 - p_j), while no earlier
 *     one has (threshold Q_i = floor(q_i 2^32)); the last channel with
 *     p > 0 fires if none before it did; after the first, each channel
 *     fires independently with its own threshold T_i = floor(p_i 2^32);
 *   - a depolarizing channel that fired takes k = min(floor(u m / U), m-1)
 *     with U the threshold that decided it (Q_i or T_i), m = 3 / 15.
 * Conditioning on "the group fired" and walking to the first fired channel
 * reproduces independent Bernoulli(p_i) channels: P(first = i | fired) =
 * prod_{j<i}(1 - p_j) p_i / (1 - R_0). */
#define OR_GROUP 32

static uint32_t stream_word(uint64_t seed, uint64_t shot, uint32_t ctr2, uint32_t tag, int w)
{
    uint32_t ctr[4] = {(uint32_t)shot, (uint32_t)(shot >> 32), ctr2, tag};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    or_philox(ctr, key, out);
    return out[w];
}

static uint32_t outcome_after(int32_t type, uint32_t u, uint32_t U)
{
    if (type != CH_DEP1 && type != CH_DEP2) return 1u;
    uint64_t m = type == CH_DEP1 ? 3u : 15u;
    uint64_t k = ((uint64_t)u * m) / U;
    if (k > m - 1) k = m - 1;
    return (uint32_t)k + 1u;
}

static void apply_outcome(const orc_prog *P, int64_t c, uint32_t v, uint64_t *b)
{
    for (int32_t i = 0; i < P->ch_nsym[c]; i++)
        if ((v >> i) & 1u) flipb(b, P->ch_sym0[c] + i);
}

void or_draw_grouped(const orc_prog *P, uint64_t seed, uint64_t shot, uint64_t *b)
{
    memset(b, 0, (size_t)P->pw * 8);
    b[0] = 1u;
    int64_t *fault = (int64_t *)malloc((size_t)(P->nch > 0 ? P->nch : 1) * sizeof(int64_t));
    if (!fault) return;
    int64_t nf = 0, r = 0;
    for (int64_t c = 0; c < P->nch; c++) {
        if (P->ch_type[c] == CH_RANDOM) {
            uint32_t w = stream_word(seed, shot, (uint32_t)(r / 128), 3u, (int)((r / 32) % 4));
            if ((w >> (r % 32)) & 1u) apply_outcome(P, c, 1u, b);
            r++;
        } else {
            fault[nf++] = c;
        }
    }
    for (int64_t g = 0; g * OR_GROUP < nf; g++) {
        int64_t n = nf - g * OR_GROUP < OR_GROUP ? nf - g * OR_GROUP : OR_GROUP;
        const int64_t *ch = fault + g * OR_GROUP;
        /* R[i] = prod_{j >= i} (1 - p_j), R[n] = 1 */
        double R[OR_GROUP + 1];
        R[n] = 1.0;
        for (int64_t i = n - 1; i >= 0; i--) R[i] = R[i + 1] * (1.0 - P->ch_p[ch[i]]);
        uint32_t G = or_threshold(1.0 - R[0]);
        uint32_t ug = stream_word(seed, shot, (uint32_t)(g / 4), 1u, (int)(g % 4));
        if (ug >= G) continue;
        int64_t last = -1;
        for (int64_t i = 0; i < n; i++)
            if (P->ch_p[ch[i]] > 0.0) last = i;
        int searching = 1;
        for (int64_t i = 0; i < n; i++) {
            int64_t c = ch[i];
            uint32_t u = stream_word(seed, shot, (uint32_t)(8 * g + i / 4), 2u, (int)(i % 4));
            uint32_t U;
            int fired;
            if (searching) {
                U = i == last ? 4294967295u : or_threshold(P->ch_p[c] / (1.0 - R[i]));
                fired = i == last || u < U;
                if (fired) searching = 0;
            } else {
                U = P->ch_T[c];
                fired = u < U;
            }
            if (fired) apply_outcome(P, c, outcome_after(P->ch_type[c], u, U), b);
        }
    }
    free(fault);
}

void or_sample_grouped(const orc_prog *P, uint64_t seed, uint64_t shot0, int64_t nshots,
                       uint64_t *meas, uint64_t *det, uint64_t *obs)
{
    int64_t wm = (P->nmeas + 63) / 64, wd = (P->ndet + 63) / 64, wo = (P->nobs + 63) / 64;
    uint64_t *b = (uint64_t *)malloc((size_t)P->pw * 8);
    if (!b) return;
    for (int64_t t = 0; t < nshots; t++) {
        or_draw_grouped(P, seed, shot0 + (uint64_t)t, b);
        or_eval(P, b, meas + t * wm, det + t * wd, obs + t * wo);
    }
    free(b);
}

/* ---------------------------------------------------------- expectation */
static int channel_outcomes(int32_t type) { return type == CH_DEP1 ? 3 : (type == CH_DEP2 ? 15 : 1); }

/* probability that the masked bits of channel c have odd parity, at rate p
 * (random channels are fair coins) */
static double odd_probability(const orc_prog *P, int64_t c, uint32_t mask, double p)
{
    int32_t type = P->ch_type[c];
    if (type == CH_RANDOM) return mask ? 0.5 : 0.0;
    int m = channel_outcomes(type);
    int odd = 0;
    for (int v = 1; v <= m; v++) odd += __builtin_popcount((unsigned)v & mask) & 1;
    return p * (double)odd / (double)m;
}

static uint32_t channel_mask(const orc_prog *P, const uint64_t *row, int64_t c)
{
    uint32_t mask = 0;
    for (int32_t i = 0; i < P->ch_nsym[c]; i++) mask |= (uint32_t)getb(row, P->ch_sym0[c] + i) << i;
    return mask;
}

static const uint64_t *target_row(const orc_prog *P, int64_t j)
{
    return j < P->ndet ? P->det + j * P->pw : P->obs + (j - P->ndet) * P->pw;
}

/* log|E_j| and sign for the ndet detectors then the nobs observables;
 * p[c] per channel (random channels ignore it) */
void or_expect(const orc_prog *P, const double *p, double *logabs, int8_t *sign)
{
    for (int64_t j = 0; j < P->ndet + P->nobs; j++) {
        const uint64_t *row = target_row(P, j);
        double acc = 0.0;
        int neg = getb(row, 0);
        for (int64_t c = 0; c < P->nch; c++) {
            uint32_t mask = channel_mask(P, row, c);
            if (!mask) continue;
            double f = 1.0 - 2.0 * odd_probability(P, c, mask, p[c]);
            if (f < 0) neg ^= 1;
            acc += log(fabs(f));
        }
        logabs[j] = acc;
        sign[j] = neg ? -1 : 1;
    }
}

/* grad_p[c] = sum_j g[j] d log|E_j| / d p_c */
void or_expect_vjp(const orc_prog *P, const double *p, const double *g, double *grad_p)
{
    for (int64_t c = 0; c < P->nch; c++) grad_p[c] = 0.0;
    for (int64_t j = 0; j < P->ndet + P->nobs; j++) {
        const uint64_t *row = target_row(P, j);
        for (int64_t c = 0; c < P->nch; c++) {
            uint32_t mask = channel_mask(P, row, c);
            if (!mask || P->ch_type[c] == CH_RANDOM) continue;
            double dP = odd_probability(P, c, mask, 1.0); /* d P(odd) / dp */
            double f = 1.0 - 2.0 * odd_probability(P, c, mask, p[c]);
            grad_p[c] += g[j] * (-2.0 * dP / f);
        }
    }
}
