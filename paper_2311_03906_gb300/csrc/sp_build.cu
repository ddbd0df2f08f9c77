// sp_build.cu -- Algorithm 1 "Initialization" on the GPU (arXiv 2311.03906).
//
// The symbolic tableau of Eq. stabilizer3 is 2n x (2n + n_s + 1) bits.  By
// Fact 2 every branch of A-G's algorithm depends only on the X/Z part, so the
// traversal runs in two passes:
//   K1 k_traverse   walks the ops over the X/Z tableau plus the constant
//                   phase column (Init-C, Fact 1, Init-M on column 0), kept
//                   qubit-major and bit-parallel over rows, in one CTA's
//                   shared memory or spread over a thread-block cluster.  It
//                   writes a log of the row operations that touch symbol
//                   columns, and each fault symbol's injection column
//                   (Init-P: X^{s} flips rows with z_a = 1, Z^{s} rows with
//                   x_a = 1);
//   K2 k_replay     every symbol column is replayed through that log from
//                   the moment its symbol appears, 32 columns per thread as
//                   bit-sliced words in shared memory.  The outcome vector of
//                   a measurement (Init-M) is the XOR of its row set.
// Only stabilizer-row phases are replayed: destabilizer phases never feed a
// stabilizer phase or an outcome in A-G's algorithm.  Detector and
// observable rows are XORs of measurement rows (K3).
#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <vector>

#include <cooperative_groups.h>

#include "sp_internal.h"

namespace sp {

constexpr int TRAV_THREADS = 1024;
constexpr uint32_t FULL = 0xffffffffu;
constexpr int REPLAY_SPLIT_MIN_N = 256;   // qubits from which k_replay runs 8 warps per CTA

__device__ __forceinline__ int gcount(uint32_t x1, uint32_t z1, uint32_t x2, uint32_t z2)
{
    // Power of i collected per qubit when the Pauli word (x1,z1) multiplies
    // (x2,z2) from the left: +1 for the cyclic pairs XY, YZ, ZX and -1 for
    // YX, ZY, XZ (A-G's g-function, summed over 32 qubits).
    uint32_t X1 = x1 & ~z1, Y1 = x1 & z1, Z1 = z1 & ~x1;
    uint32_t X2 = x2 & ~z2, Y2 = x2 & z2, Z2 = z2 & ~x2;
    uint32_t pos = (X1 & Y2) | (Y1 & Z2) | (Z1 & X2);
    uint32_t neg = (X1 & Z2) | (Y1 & X2) | (Z1 & Y2);
    return __popc(pos) - __popc(neg);
}

__device__ __forceinline__ int warp_sum(int v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// One step of the traversal: a group of ops on disjoint qubits (gates and
// noise injections, run in parallel) or one barrier op (a measurement, reset
// or feed-forward, run by the whole CTA).  Ops are sched[begin, end).
struct TravStep {
    uint32_t begin, end;
    uint32_t barrier;
    uint32_t inj_before;    // noise ops before this step in circuit order
    uint32_t fsym_before;   // fault symbols before this step
    uint32_t pad[3];
};

struct TravParams {
    const Inst *insts;
    const uint32_t *sched;
    const TravStep *steps;
    int64_t nsteps;
    uint32_t ninj_total, nfsym_total;
    int n, SW;               // qubits; 32-row words per column
    uint32_t *gtab;          // used when the tableau does not fit in shared memory
    int tab_in_smem;
    uint32_t *log;
    uint64_t log_cap;
    uint32_t *inj;           // [(cap_sym + 2) * SW]
    uint64_t *sym_logpos;    // [cap_sym + 2]
    uint8_t *sym_random;     // [cap_sym + 2]
    uint32_t *chT;
    uint8_t *chKind;
    uint32_t *chSym0;
    float *chP;
    uint8_t *rec_const;
    uint64_t *ev_pos;        // log positions of the events other than injections
    uint64_t ev_cap;
    TraverseCounts *counts;
    int qp;                  // qubits per CTA of a cluster
};

constexpr int TAB_XS = 0, TAB_ZS = 1, TAB_XD = 2, TAB_ZD = 3;

// Bit i of the result = XOR of bits 0..i-1 of x.
__device__ __forceinline__ uint32_t prefix_xor_excl(uint32_t x)
{
    uint32_t y = x << 1;
    y ^= y << 1;
    y ^= y << 2;
    y ^= y << 4;
    y ^= y << 8;
    y ^= y << 16;
    return y;
}

// One warp writes the rows of the mask words (lane = word; lanes past the
// last word pass 0) to dst in increasing order and returns their number.
__device__ __forceinline__ uint32_t write_rows(uint32_t *dst, uint32_t m, int lane)
{
    const uint32_t c = __popc(m);
    uint32_t inc = c;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    const uint32_t total = __shfl_sync(FULL, inc, 31);
    uint32_t off = inc - c;
    while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        dst[off++] = 32u * (uint32_t)lane + (uint32_t)b;
    }
    return total;
}

// K1: the X/Z pass, qubit-major.  The tableau is kept per qubit q as four
// bit-vectors over the n stabilizer rows (32 rows per word): XS(q), ZS(q) of
// the stabilizers and XD(q), ZD(q) of the destabilizers (destabilizer i pairs
// with stabilizer i), plus the stabilizer phases r as one bit-vector.  A gate
// (Init-C's column rules, Fact 1 for Paulis) is a few word operations per 32
// rows, an injection column (Init-P: X^s flips the rows with z_q = 1, Z^s the
// rows with x_q = 1) is a column read, and a measurement (Init-M) works on
// whole columns.  Gates and injections arrive in groups on disjoint qubits,
// one op per warp at a time with lane = row word; a gate's phase flips stay
// in the lane's register until the next barrier.  Measurements, resets and
// feed-forward ops are barriers.
//
// CL > 1: a cluster of CL CTAs, CTA r holding the columns of qubits
// [r*QP, (r+1)*QP) in its shared memory (other CTAs' columns through
// distributed shared memory).  Each CTA applies the ops on its own qubits and
// the row operations of a measurement to its own columns; rank 0 keeps the
// phases (changed only by atomic XORs), combines the CTAs' partial phase
// counts and writes the log.  Values every CTA needs (the pivot, the row
// masks and their counts) are computed by each from the measured column, so
// all CTAs keep the same log position.  Requires n <= 1024.
template <int CL>
__global__ void __launch_bounds__(TRAV_THREADS, 1) k_traverse(TravParams P)
{
    extern __shared__ __align__(16) uint32_t tsm[];
    __shared__ uint32_t s_rs[32], s_m0[32], s_m1[32], s_za[32], s_px[32], s_pz[32];
    __shared__ uint32_t s_c0[32 * 32], s_c1[32 * 32];
    __shared__ uint32_t s_gc0[CL * 32], s_gc1[CL * 32];   // rank 0: the CTAs' phase counts
    __shared__ int s_gG[CL];                              // rank 0: the CTAs' power-of-i sums
    __shared__ int s_red[32];
    __shared__ int s_p, s_e, s_err;
    __shared__ uint32_t s_cnt;
    namespace cg = cooperative_groups;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int n = P.n, SW = P.SW;
    // a qubit's four bit-vectors plus one pad word: an odd stride, so that
    // threads reading one word of consecutive qubits hit distinct banks
    const int QSTR = 4 * SW + 1;
    int rank = 0, q0 = 0, nq = n;
    uint32_t *tab = P.tab_in_smem ? tsm : P.gtab;
    if constexpr (CL > 1) {
        rank = (int)cg::this_cluster().block_rank();
        q0 = rank * P.qp;
        nq = max(0, min(P.qp, n - q0));
        tab = tsm;
    }
    // rank 0's copy of a shared array (this CTA's own for CL = 1)
    auto at0 = [&](auto *x) {
        if constexpr (CL > 1) return cg::this_cluster().map_shared_rank(x, 0);
        else return x;
    };
    auto csync = [&]() {
        if constexpr (CL > 1) cg::this_cluster().sync();
        else __syncthreads();
    };
    // column of qubit q (in another CTA's shared memory for CL > 1)
    auto col = [&](int q) -> uint32_t * {
        if constexpr (CL > 1) {
            const int o = q / P.qp;
            uint32_t *base = o == rank ? tsm : cg::this_cluster().map_shared_rank(tsm, o);
            return base + (size_t)(q - o * P.qp) * QSTR;
        } else {
            return tab + (size_t)q * QSTR;
        }
    };
    auto own = [&](int q) { return CL == 1 || q / P.qp == rank; };

    // stabilizer i = Z_i, destabilizer i = X_i, phases 0
    for (int64_t i = t; i < (int64_t)nq * QSTR; i += TRAV_THREADS) {
        const int q = q0 + (int)(i / QSTR), r = (int)(i % QSTR), k = r / SW, w = r % SW;
        tab[i] = ((k == TAB_ZS || k == TAB_XD) && w == (q >> 5)) ? 1u << (q & 31) : 0u;
    }
    if (t < 32) s_rs[t] = 0;
    if (t == 0) s_err = 0;
    csync();

    uint32_t rd = 0;                     // this lane's pending phase flips
    uint32_t nrand = 0, nrec = 0, inj_mark = 0, err = 0, nev = 0;
    // every event other than an injection is also listed by position
    auto note_event = [&](uint64_t at) {
        if (t == 0 && rank == 0 && nev < P.ev_cap) P.ev_pos[nev] = at;
        nev++;
    };
    uint64_t lp = 0;                     // log position after the last barrier's event
    for (int64_t si = 0; si < P.nsteps; si++) {
        const TravStep S = P.steps[si];
        if (!S.barrier) {
            for (uint32_t k = S.begin + (uint32_t)warp; k < S.end; k += TRAV_THREADS / 32) {
                const Inst in = P.insts[P.sched[k]];
                const uint32_t code = in.code;
                if (!own((int)in.a)) continue;
                if (code <= I_Z) {
                    if (lane >= SW) continue;
                    uint32_t *ca = col((int)in.a);
                    uint32_t *XS = ca + TAB_XS * SW + lane, *ZS = ca + TAB_ZS * SW + lane;
                    uint32_t *XD = ca + TAB_XD * SW + lane, *ZD = ca + TAB_ZD * SW + lane;
                    switch (code) {
                    case I_H: {
                        const uint32_t xs = *XS, zs = *ZS, xd = *XD, zd = *ZD;
                        rd ^= xs & zs;
                        *XS = zs; *ZS = xs; *XD = zd; *ZD = xd;
                    } break;
                    case I_S: {
                        const uint32_t xs = *XS, zs = *ZS;
                        rd ^= xs & zs;
                        *ZS = zs ^ xs;
                        *ZD ^= *XD;
                    } break;
                    case I_X: rd ^= *ZS; break;
                    case I_Z: rd ^= *XS; break;
                    case I_Y: rd ^= *XS ^ *ZS; break;
                    case I_CX: {
                        uint32_t *cb = col((int)in.b);
                        const uint32_t xa = *XS, za = *ZS;
                        const uint32_t xb = cb[TAB_XS * SW + lane], zb = cb[TAB_ZS * SW + lane];
                        rd ^= xa & zb & ~(xb ^ za);
                        cb[TAB_XS * SW + lane] = xb ^ xa;
                        *ZS = za ^ zb;
                        cb[TAB_XD * SW + lane] ^= *XD;
                        *ZD ^= cb[TAB_ZD * SW + lane];
                    } break;
                    default: break;
                    }
                    continue;
                }
                // Init-P: the injection column of each symbol over the
                // stabilizer rows; log slots in circuit order
                const int kk = code == I_DEP2 ? 4 : (code == I_DEP1 ? 2 : 1);
                const uint32_t s0 = 1u + in.sym_base + nrand, ch = in.gi + nrand;
                const uint64_t slot = lp + 2ull * (in.gi - inj_mark);
                if (slot + 2 > P.log_cap) {
                    s_err = 1;
                    continue;
                }
                for (int j = 0; j < kk; j++) {
                    const uint32_t q = (j < 2) ? in.a : in.b;
                    bool useZ, useX;
                    if (code == I_XERR) { useZ = true; useX = false; }
                    else if (code == I_ZERR) { useZ = false; useX = true; }
                    else if (code == I_YERR) { useZ = true; useX = true; }
                    else { useZ = !(j & 1); useX = (j & 1) != 0; }
                    if (lane < SW) {
                        const uint32_t *cq = col((int)q);
                        uint32_t v = 0;
                        if (useZ) v ^= cq[TAB_ZS * SW + lane];
                        if (useX) v ^= cq[TAB_XS * SW + lane];
                        P.inj[(size_t)(s0 + j) * SW + lane] = v;
                    }
                    if (lane == 0) {
                        P.sym_logpos[s0 + j] = slot;
                        P.sym_random[s0 + j] = 0;
                    }
                }
                if (lane == 0) {
                    P.chT[ch] = in.aux;
                    P.chP[ch] = __uint_as_float(in.pbits);
                    P.chKind[ch] = (kk == 1) ? CK_BERN : (kk == 2 ? CK_DEP1 : CK_DEP2);
                    P.chSym0[ch] = s0;
                    P.log[slot] = (EV_INJECT << 24) | (uint32_t)kk;
                    P.log[slot + 1] = s0;
                }
            }
            csync();
            continue;
        }
        // ---- barrier op ------------------------------------------------------
        // Every column is final here (the last group or barrier step ended
        // with a cluster barrier).  Pending phase flips go to rank 0 now; rank
        // 0 reads its phases only after the next cluster barrier.
        lp += 2ull * (S.inj_before - inj_mark);   // the segment's injection events
        inj_mark = S.inj_before;
        if (lane < SW && rd) atomicXor(at0(s_rs) + lane, rd);
        rd = 0;
        const Inst in = P.insts[P.sched[S.begin]];
        const uint32_t code = in.code;
        const int a = (int)in.a;
        if (lp + 2 * (uint64_t)n + 8 > P.log_cap || nev + 2 > P.ev_cap) { err = 1; break; }
        uint32_t *ca = col(a);
        const bool own_a = own(a);
        if (code >= I_XIF) {
            // Feed-forward (the conditional Paulis of Sec. 6): P^e on qubit a
            // with e the form of record in.b.  A stabilizer that
            // anticommutes with P (X: z_a, Z: x_a, Y: x_a ^ z_a) gets e: its
            // constant bit here, its symbol part in the replay (EV_FF).
            if (warp == 0) {
                const bool useZ = code != I_ZIF, useX = code != I_XIF;
                uint32_t m = 0;
                if (lane < SW) {
                    if (useZ) m ^= ca[TAB_ZS * SW + lane];
                    if (useX) m ^= ca[TAB_XS * SW + lane];
                }
                const uint32_t total = (uint32_t)warp_sum(__popc(m));
                if (rank == 0) {
                    write_rows(P.log + lp + 2, m, lane);
                    if (P.rec_const[in.b] && m) atomicXor(&s_rs[lane], m);
                    if (lane == 0) {
                        P.log[lp] = (EV_FF << 24) | total;
                        P.log[lp + 1] = in.b;
                    }
                }
                if (lane == 0) s_cnt = total;
            }
            __syncthreads();
            note_event(lp);
            lp += 2 + (uint64_t)s_cnt;
            csync();   // every CTA has read the column before the next step changes it
            continue;
        }
        // ---- Init-M (M, MR, R) -----------------------------------------------
        const bool recorded = (code != I_R), reset = (code != I_M);
        const uint32_t rec = recorded ? nrec : NO_REC;
        if (warp == 0) {
            // the measured column, read by every CTA before anyone changes it:
            // the first stabilizer with x_a = 1 (if any), the row masks, z_a
            const uint32_t xw = lane < SW ? ca[TAB_XS * SW + lane] : 0u;
            const uint32_t bal = __ballot_sync(FULL, xw != 0u);
            int p = -1;
            if (bal) {
                const int L = __ffs(bal) - 1;
                p = 32 * L + __ffs(__shfl_sync(FULL, xw, L)) - 1;
            }
            s_m0[lane] = p >= 0 && lane == (p >> 5) ? xw & ~(1u << (p & 31)) : xw;   // stabilizers (random case)
            s_m1[lane] = lane < SW ? ca[TAB_XD * SW + lane] : 0u;                     // destabilizers
            s_za[lane] = lane < SW ? ca[TAB_ZS * SW + lane] : 0u;
            if (lane == 0) s_p = p;
        }
        __syncthreads();
        const int p = s_p;
        uint32_t e_const = 0;
        uint32_t zpa = 0;   // z_a of the pivot (random outcomes)
        if (p >= 0) {
            // random outcome: every other row with x_a = 1 becomes P_p * row
            const int wp = p >> 5;
            const uint32_t bp = 1u << (p & 31);
            zpa = (s_za[wp] & bp) ? 1u : 0u;
            const int la = own_a ? a - q0 : -1;   // the measured column, if this CTA holds it
            {
                // the pivot stabilizer on this CTA's qubits, one bit per qubit
                uint32_t xp = 0, zp = 0;
                if (t < nq) {
                    const uint32_t *cq = tab + (size_t)t * QSTR;
                    xp = (cq[TAB_XS * SW + wp] & bp) ? 1u : 0u;
                    zp = (cq[TAB_ZS * SW + wp] & bp) ? 1u : 0u;
                }
                const uint32_t bx = __ballot_sync(FULL, xp), bz = __ballot_sync(FULL, zp);
                if (lane == 0) {
                    s_px[warp] = bx;
                    s_pz[warp] = bz;
                }
            }
            __syncthreads();
            // Rowsum of every masked row with the pivot on this CTA's columns,
            // one column per warp at a time.  For the stabilizer rows, A-G's
            // power of i (g summed over the qubits) is counted mod 4 in
            // bit-sliced form (c1 c0).  The measured column is counted here
            // but written only after the next cluster barrier, when every CTA
            // is done reading it.
            uint32_t c0 = 0, c1 = 0;
            if (lane < SW) {
                const uint32_t ms = s_m0[lane], md = s_m1[lane];
                // two columns at a time: their words are read before any is
                // written, so the loads overlap (distinct qubits never alias)
                constexpr int QB = 2, QS = TRAV_THREADS / 32;
                for (int l0 = warp; l0 < nq; l0 += QB * QS) {
                    uint32_t xq[QB], zq[QB], xs[QB], zs[QB], xd[QB], zd[QB];
#pragma unroll
                    for (int u = 0; u < QB; u++) {
                        const int l = l0 + u * QS;
                        xq[u] = l < nq ? (s_px[l >> 5] >> (l & 31)) & 1u : 0u;
                        zq[u] = l < nq ? (s_pz[l >> 5] >> (l & 31)) & 1u : 0u;
                        xs[u] = zs[u] = xd[u] = zd[u] = 0u;
                        if (xq[u] | zq[u]) {
                            const uint32_t *cq = tab + (size_t)l * QSTR;
                            xs[u] = cq[TAB_XS * SW + lane];
                            zs[u] = cq[TAB_ZS * SW + lane];
                            if (md && xq[u]) xd[u] = cq[TAB_XD * SW + lane];
                            if (md && zq[u]) zd[u] = cq[TAB_ZD * SW + lane];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < QB; u++) {
                        if (!(xq[u] | zq[u])) continue;
                        const uint32_t X2 = xs[u] & ~zs[u], Y2 = xs[u] & zs[u], Z2 = zs[u] & ~xs[u];
                        // +1 for the pairs (pivot, row) = XY, YZ, ZX; -1 for YX, ZY, XZ
                        uint32_t pos, neg;
                        if (xq[u] && !zq[u]) { pos = Y2; neg = Z2; }
                        else if (xq[u]) { pos = Z2; neg = X2; }
                        else { pos = X2; neg = Y2; }
                        pos &= ms;
                        neg &= ms;
                        c1 ^= c0 & pos;
                        c0 ^= pos;
                        c1 ^= ~c0 & neg;
                        c0 ^= neg;
                        if (l0 + u * QS == la) continue;   // the measured column: later
                        uint32_t *cq = tab + (size_t)(l0 + u * QS) * QSTR;
                        if (xq[u]) cq[TAB_XS * SW + lane] = xs[u] ^ ms;
                        if (zq[u]) cq[TAB_ZS * SW + lane] = zs[u] ^ ms;
                        if (md) {
                            if (xq[u]) cq[TAB_XD * SW + lane] = xd[u] ^ md;
                            if (zq[u]) cq[TAB_ZD * SW + lane] = zd[u] ^ md;
                        }
                    }
                }
            }
            s_c0[warp * 32 + lane] = c0;
            s_c1[warp * 32 + lane] = c1;
            __syncthreads();
            // destabilizer p := the old stabilizer p; stabilizer p := Z_a (the
            // measured column later)
            if (t < nq && t != la) {
                uint32_t *cq = tab + (size_t)t * QSTR;
                const bool xp = (s_px[t >> 5] >> (t & 31)) & 1u, zp = (s_pz[t >> 5] >> (t & 31)) & 1u;
                cq[TAB_XD * SW + wp] = (cq[TAB_XD * SW + wp] & ~bp) | (xp ? bp : 0u);
                cq[TAB_ZD * SW + wp] = (cq[TAB_ZD * SW + wp] & ~bp) | (zp ? bp : 0u);
                cq[TAB_XS * SW + wp] &= ~bp;
                cq[TAB_ZS * SW + wp] &= ~bp;
            }
            if (warp == 0) {
                // this CTA's mod-4 counts, to rank 0
                uint32_t a0 = 0, a1 = 0;
                for (int w = 0; w < TRAV_THREADS / 32; w++) {
                    const uint32_t b0 = s_c0[w * 32 + lane], b1 = s_c1[w * 32 + lane];
                    a1 ^= b1 ^ (a0 & b0);
                    a0 ^= b0;
                }
                at0(s_gc0)[rank * 32 + lane] = a0;
                at0(s_gc1)[rank * 32 + lane] = a1;
                const uint32_t ms = lane < SW ? s_m0[lane] : 0u;
                const uint32_t total = (uint32_t)warp_sum(__popc(ms));
                if (lane == 0) s_cnt = total;
            }
            csync();   // counts and phase flips gathered; nobody reads the measured column any more
            if (la >= 0 && warp == 0 && lane < SW) {
                // the measured column: rowsum (the pivot has x_a = 1), then
                // row p := the old stabilizer p (destabilizer) and Z_a (stabilizer)
                uint32_t *cq = tab + (size_t)la * QSTR;
                const uint32_t ms = s_m0[lane], md = s_m1[lane];
                uint32_t xs = cq[TAB_XS * SW + lane] ^ ms, zs = cq[TAB_ZS * SW + lane] ^ (zpa ? ms : 0u);
                uint32_t xd = cq[TAB_XD * SW + lane] ^ md, zd = cq[TAB_ZD * SW + lane] ^ (zpa ? md : 0u);
                if (lane == wp) {
                    xd |= bp;
                    zd = zpa ? (zd | bp) : (zd & ~bp);
                    xs &= ~bp;
                    zs |= bp;
                }
                cq[TAB_XS * SW + lane] = xs;
                cq[TAB_ZS * SW + lane] = zs;
                cq[TAB_XD * SW + lane] = xd;
                cq[TAB_ZD * SW + lane] = zd;
            }
            if (rank == 0 && warp == 0) {
                uint32_t a0 = 0, a1 = 0;
                for (int r = 0; r < CL; r++) {
                    const uint32_t b0 = s_gc0[r * 32 + lane], b1 = s_gc1[r * 32 + lane];
                    a1 ^= b1 ^ (a0 & b0);
                    a0 ^= b0;
                }
                const uint32_t ms = lane < SW ? s_m0[lane] : 0u;
                if (a0 & ms) s_err = 2;
                // new r = r ^ r_p ^ (power of i) / 2 on the masked rows; r_p := 0
                const uint32_t rp = __shfl_sync(FULL, lane < SW ? s_rs[lane] : 0u, wp) & bp ? 1u : 0u;
                uint32_t flip = ms & (a1 ^ (rp ? FULL : 0u));
                if (lane == wp && rp) flip ^= bp;
                if (lane < SW && flip) atomicXor(&s_rs[lane], flip);
                const uint32_t total = write_rows(P.log + lp + 4, ms, lane);
                if (lane == 0) {
                    const uint32_t s = 1u + S.fsym_before + nrand, ch = S.inj_before + nrand;
                    P.log[lp] = (EV_MRAND << 24) | total;
                    P.log[lp + 1] = (uint32_t)p;
                    P.log[lp + 2] = s;
                    P.log[lp + 3] = rec;
                    P.chT[ch] = 0x80000000u;
                    P.chP[ch] = 0.5f;
                    P.chKind[ch] = CK_RANDOM;
                    P.chSym0[ch] = s;
                    P.sym_logpos[s] = lp;
                    P.sym_random[s] = 1;
                }
            }
            note_event(lp);
            lp += 4 + (uint64_t)s_cnt;
            nrand++;
        } else {
            // deterministic outcome: the product of the stabilizers paired with
            // destabilizers that have x_a = 1.  Its power of i is a sum over
            // qubits: thread q multiplies the rows' single-qubit Paulis in row
            // order, 32 rows at a time (exclusive prefix XOR = the product of
            // the earlier rows), with A-G's g-function per row.
            int G = 0;
            if (t < nq) {
                const uint32_t *cq = tab + (size_t)t * QSTR;
                uint32_t cx = 0, cz = 0;
                for (int w = 0; w < SW; w++) {
                    const uint32_t d = s_m1[w];
                    if (!d) continue;
                    const uint32_t xs = cq[TAB_XS * SW + w] & d, zs = cq[TAB_ZS * SW + w] & d;
                    if (!(xs | zs)) continue;
                    const uint32_t px = prefix_xor_excl(xs) ^ (cx ? FULL : 0u);
                    const uint32_t pz = prefix_xor_excl(zs) ^ (cz ? FULL : 0u);
                    G += gcount(xs, zs, px, pz);
                    cx ^= __popc(xs) & 1u;
                    cz ^= __popc(zs) & 1u;
                }
            }
            G = warp_sum(G);
            if (lane == 0) s_red[warp] = G;
            __syncthreads();
            if (warp == 0) {
                const int g = warp_sum(s_red[lane]);
                const uint32_t d = lane < SW ? s_m1[lane] : 0u;
                const uint32_t total = (uint32_t)warp_sum(__popc(d));
                if (lane == 0) {
                    at0(s_gG)[rank] = g;
                    s_cnt = total;
                }
            }
            csync();   // the sums and phase flips gathered
            if (rank == 0 && warp == 0) {
                const uint32_t d = lane < SW ? s_m1[lane] : 0u;
                const int g = warp_sum(lane < CL ? s_gG[lane] : 0) +
                              2 * warp_sum(__popc(lane < SW ? (s_rs[lane] & d) : 0u));
                write_rows(P.log + lp + 2, d, lane);
                if (lane == 0) {
                    const int tot = g & 3;
                    s_e = (tot == 2) ? 1 : 0;
                    if (tot & 1) s_err = 2;
                    P.log[lp] = (EV_MDET << 24) | s_cnt;
                    P.log[lp + 1] = rec;
                }
            }
            __syncthreads();
            note_event(lp);
            lp += 2 + (uint64_t)s_cnt;
            e_const = rank == 0 ? (uint32_t)s_e : 0u;
        }
        if (recorded) {
            if (t == 0 && rank == 0) P.rec_const[nrec] = (uint8_t)e_const;
            nrec++;
        }
        if (reset) {
            // conditional X^e on qubit a: flip every stabilizer with z_a = 1
            // after the measurement (a random outcome changed z_a on the
            // masked rows by the pivot's z_a, and row p is Z_a)
            if (warp == 0) {
                uint32_t m = lane < SW ? s_za[lane] : 0u;
                if (p >= 0 && lane < SW) {
                    if (zpa) m ^= s_m0[lane];
                    if (lane == (p >> 5)) m |= 1u << (p & 31);
                }
                const uint32_t total = (uint32_t)warp_sum(__popc(m));
                if (rank == 0) {
                    write_rows(P.log + lp + 1, m, lane);
                    if (e_const && m) atomicXor(&s_rs[lane], m);
                    if (lane == 0) P.log[lp] = (EV_RESET << 24) | total;
                }
                if (lane == 0) s_cnt = total;
            }
            __syncthreads();
            note_event(lp);
            lp += 1 + (uint64_t)s_cnt;
        }
        csync();   // the measured column written; the next step may read it
    }
    if (!err) lp += 2ull * (P.ninj_total - inj_mark);   // the last segment's injections
    csync();
    if (t == 0 && rank == 0) {
        uint32_t e2 = (uint32_t)s_err;
        if constexpr (CL > 1)
            for (int r = 1; r < CL; r++) e2 = max(e2, (uint32_t)*cg::this_cluster().map_shared_rank(&s_err, r));
        P.counts->log_len = lp;
        P.counts->nsym = P.nfsym_total + nrand;
        P.counts->nch = P.ninj_total + nrand;
        P.counts->nrec = nrec;
        P.counts->nev = nev;
        P.counts->err = err ? err : e2;
    }
    csync();   // no CTA leaves while another may still read its shared memory
}

// v[i][lane] ^= x for the rows of one logged event.  The rows of an event
// are distinct (a scan over the tableau's rows), so eight of them are read
// before any is written: the shared-memory round trips and the loads of the
// row indices overlap instead of running one after another.  A warp whose
// lanes all have x = 0 skips the event.
__device__ __forceinline__ void replay_xor_rows(uint32_t *v, const uint32_t *__restrict__ rows, uint32_t cnt, int n,
                                                int lane, uint32_t x)
{
    if (!__any_sync(0xffffffffu, x != 0u)) return;
    uint32_t j = 0;
    for (; j + 8 <= cnt; j += 8) {
        uint32_t i[8], a[8];
#pragma unroll
        for (int k = 0; k < 8; k++) i[k] = rows[j + k];
#pragma unroll
        for (int k = 0; k < 8; k++) a[k] = i[k] < (uint32_t)n ? v[i[k] * 32 + lane] : 0u;
#pragma unroll
        for (int k = 0; k < 8; k++)
            if (i[k] < (uint32_t)n) v[i[k] * 32 + lane] = a[k] ^ x;
    }
    for (; j < cnt; j++) {
        const uint32_t i = rows[j];
        if (i < (uint32_t)n) v[i * 32 + lane] ^= x;
    }
}

// XOR of v[i][lane] over the rows of one logged event (rows past n read row
// n-1, as a malformed log must not leave the table).
__device__ __forceinline__ uint32_t replay_xor_of_rows(const uint32_t *v, const uint32_t *__restrict__ rows,
                                                       uint32_t cnt, int n, int lane)
{
    uint32_t acc[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    uint32_t j = 0;
    for (; j + 8 <= cnt; j += 8) {
        uint32_t i[8];
#pragma unroll
        for (int k = 0; k < 8; k++) i[k] = min(rows[j + k], (uint32_t)n - 1u);
#pragma unroll
        for (int k = 0; k < 8; k++) acc[k] ^= v[i[k] * 32 + lane];
    }
    for (; j < cnt; j++) acc[0] ^= v[min(rows[j], (uint32_t)n - 1u) * 32 + lane];
    return ((acc[0] ^ acc[1]) ^ (acc[2] ^ acc[3])) ^ ((acc[4] ^ acc[5]) ^ (acc[6] ^ acc[7]));
}

// K2: column-parallel replay.  A CTA of NW warps owns 1024 symbols: lane l
// holds symbols 32*(32*blockIdx + l) .. +31 as one bit-sliced word per
// stabilizer row, in a table v[n][32] shared by the warps.  The CTA walks the
// log's events other than injections (ev_pos, from the first one at or after
// its first symbol); before each it injects its own fault symbols whose
// injection came earlier (sym_logpos; injections after the last event reach
// no record).  The warps split each event's row list; an event that changes
// the table ends with a barrier.  Every skip decision depends only on values
// all warps read alike (log words, the table before the event, the symbols),
// so the barriers are uniform across the CTA.
template <int NW>
__global__ void __launch_bounds__(32 * NW, 1) k_replay(const uint32_t *__restrict__ log, uint64_t log_len,
                                                     const uint64_t *__restrict__ ev_pos, uint32_t nev,
                                                     const uint32_t *__restrict__ inj, int Wq,
                                                     const uint64_t *__restrict__ sym_logpos,
                                                     const uint8_t *__restrict__ sym_random, uint32_t nsym,
                                                     int n, uint32_t *__restrict__ A, int64_t apitch)
{
    extern __shared__ uint32_t v[];  // [n][32], then [NW][32] partial XORs
    uint32_t *s_acc = v + (size_t)n * 32;
    // the next 32 events: position and first four log words, loaded together
    __shared__ uint64_t s_epos[32];
    __shared__ uint4 s_ew[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t g = (int64_t)blockIdx.x * 32 + lane;
    const uint32_t blo = (uint32_t)blockIdx.x * 1024u, bhi = blo + 1024u;
    const uint32_t s_first = blo == 0 ? 1u : blo;
    if (s_first > nsym) return;
    const uint32_t s_end = min(bhi, nsym + 1u);
    for (int i = warp; i < n; i += NW) v[i * 32 + lane] = 0;
    __syncthreads();
    const uint32_t lo = (uint32_t)g * 32u, hi = lo + 32u;
    const bool write = g < apitch && warp == 0;   // warp 0 writes the records
    // the first event at or after this CTA's first symbol
    const uint64_t p0 = sym_logpos[s_first];
    uint32_t k = 0, khi = nev;
    while (k < khi) {
        const uint32_t mid = (k + khi) >> 1;
        if (ev_pos[mid] < p0) k = mid + 1; else khi = mid;
    }
    const uint32_t khi0 = k;   // batches of 32 events start here
    uint32_t s_next = s_first;
    uint32_t e = 0;
    // this warp's contiguous share of an event's cnt rows
    auto share = [&](uint32_t cnt, uint32_t &j0) {
        j0 = (uint32_t)((uint64_t)warp * cnt / NW);
        return (uint32_t)((uint64_t)(warp + 1) * cnt / NW) - j0;
    };
    for (; k < nev; k++) {
        const uint32_t kb = (k - khi0) & 31u;
        if (kb == 0) {
            __syncthreads();   // every warp is done with the previous batch
            if (warp == 0) {
                uint64_t ep = log_len;
                uint4 w = make_uint4(0u, 0u, 0u, 0u);
                if (k + lane < nev) {
                    ep = ev_pos[k + lane];
                    if (ep < log_len) w.x = log[ep];
                    if (ep + 1 < log_len) w.y = log[ep + 1];
                    if (ep + 2 < log_len) w.z = log[ep + 2];
                    if (ep + 3 < log_len) w.w = log[ep + 3];
                }
                s_epos[lane] = ep;
                s_ew[lane] = w;
            }
            __syncthreads();
        }
        const uint64_t pos = s_epos[kb];
        const uint4 ew = s_ew[kb];
        if (pos >= log_len) break;
        // Init-P for this CTA's fault symbols injected before the event: lane
        // l takes its own symbols, warps split the rows of each column
        const uint32_t s_a = s_next;
        while (s_next < s_end && sym_logpos[s_next] < pos) s_next++;
        if (s_next > s_a) {
            const uint32_t l1 = min(s_next, hi);
            for (uint32_t s = max(s_a, lo); s < l1; s++) {
                if (sym_random[s]) continue;
                const uint32_t bit = 1u << (s & 31);
                const uint32_t *col = inj + (size_t)s * Wq;
                for (int w = warp; w < Wq; w += NW) {
                    uint32_t m = col[w];
                    while (m) {
                        const int b = __ffs(m) - 1;
                        m &= m - 1;
                        if (w * 32 + b < n) v[(w * 32 + b) * 32 + lane] ^= bit;
                    }
                }
            }
            __syncthreads();
        }
        const uint32_t h = ew.x;
        const uint32_t ev = h >> 24, cnt = h & 0xffffffu;
        // every event must fit in the log and name rows below n
        const uint64_t len = ev == EV_MRAND ? 4 + (uint64_t)cnt
                           : (ev == EV_MDET || ev == EV_FF) ? 2 + (uint64_t)cnt : 1 + (uint64_t)cnt;
        if (pos + len > log_len) break;
        uint32_t j0;
        if (ev == EV_MRAND) {
            const uint32_t p = min(ew.y, (uint32_t)n - 1u), s = ew.z, rec = ew.w;
            const uint32_t vp = v[p * 32 + lane];
            e = (s >= lo && s < hi) ? (1u << (s & 31)) : 0u;
            // nothing to do when row p is zero and the new symbol is not ours
            if (__any_sync(0xffffffffu, vp != 0u) || (s >= blo && s < bhi)) {
                const uint32_t m = share(cnt, j0);
                replay_xor_rows(v, log + pos + 4 + j0, m, n, lane, vp);
                __syncthreads();   // every warp has read row p
                if (warp == 0) v[p * 32 + lane] = e;
                if (rec != NO_REC && write) A[(size_t)rec * apitch + g] = e;
                __syncthreads();
            }
        } else if (ev == EV_MDET) {
            const uint32_t rec = ew.y;
            const uint32_t m = share(cnt, j0);
            s_acc[warp * 32 + lane] = replay_xor_of_rows(v, log + pos + 2 + j0, m, n, lane);
            __syncthreads();
            e = 0;
#pragma unroll
            for (int w = 0; w < NW; w++) e ^= s_acc[w * 32 + lane];
            if (rec != NO_REC && write) A[(size_t)rec * apitch + g] = e;
            __syncthreads();   // the partials are reused by the next event
        } else if (ev == EV_FF) {
            // the record's symbol word for this lane: written earlier by
            // warp 0 (a barrier since), or still zero if the record precedes
            // its symbols
            const uint32_t rec = ew.y;
            const uint32_t ef = g < apitch ? A[(size_t)rec * apitch + g] : 0u;
            if (__any_sync(0xffffffffu, ef != 0u)) {
                const uint32_t m = share(cnt, j0);
                replay_xor_rows(v, log + pos + 2 + j0, m, n, lane, ef);
                __syncthreads();
            }
        } else if (ev == EV_RESET) {
            if (__any_sync(0xffffffffu, e != 0u)) {
                const uint32_t m = share(cnt, j0);
                replay_xor_rows(v, log + pos + 1 + j0, m, n, lane, e);
                __syncthreads();
            }
        }
    }
}

__global__ void k_merge_const(uint32_t *A, int64_t apitch, const uint8_t *rec_const, int64_t nrec)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nrec && rec_const[k]) A[(size_t)k * apitch] |= 1u;
}

// K3: detector / observable rows as XORs of measurement rows.
// One block per output row, threads over the row's words.
__global__ void k_xor_rows(uint32_t *A, int64_t apitch, const uint32_t *__restrict__ off,
                           const uint32_t *__restrict__ refs, int64_t nout, int64_t out_row0)
{
    const int64_t j = blockIdx.x;
    if (j >= nout) return;
    for (int64_t w = threadIdx.x; w < apitch; w += blockDim.x) {
        uint32_t acc = 0;
        for (uint32_t k = off[j]; k < off[j + 1]; k++) acc ^= A[(size_t)refs[k] * apitch + w];
        A[(size_t)(out_row0 + j) * apitch + w] = acc;
    }
}

__global__ void k_check_random(const uint32_t *A, int64_t apitch, int64_t row0, int64_t nrows,
                               const uint32_t *mask, int *bad)
{
    const int64_t j = blockIdx.x;
    if (j >= nrows) return;
    bool hit = false;
    for (int64_t w = threadIdx.x; w < apitch; w += blockDim.x)
        if (A[(size_t)(row0 + j) * apitch + w] & mask[w]) hit = true;
    if (__syncthreads_or(hit) && threadIdx.x == 0) atomicMin(bad, (int)j);
}

// Row nonzeros (symbols only) of A_j, or of A_j ^ A_parent(j) when parent
// is given; in fill mode the symbol indices (s-1) are written in order.
// One warp per row, four consecutive words per lane (the row pitch is a
// multiple of four words), so that each warp keeps 512 bytes of the row in
// flight: the pass streams the whole coefficient matrix.
__global__ void k_row_csr(const uint32_t *__restrict__ A, int64_t apitch, int64_t nrows,
                          const int32_t *__restrict__ parent, uint32_t *count,
                          const uint32_t *__restrict__ off, uint32_t *idx)
{
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= nrows) return;
    const uint32_t *rj = A + (size_t)j * apitch;
    const int32_t pj = parent ? parent[j] : -1;
    const uint32_t *rp = pj >= 0 ? A + (size_t)pj * apitch : nullptr;
    uint32_t base = idx ? off[j] : 0u;
    uint32_t cnt = 0;
    for (int64_t w0 = 0; w0 < apitch; w0 += 128) {
        const int64_t w = w0 + 4 * lane;
        uint32_t m[4] = {0u, 0u, 0u, 0u};
        if (w < apitch) {
            const uint4 a = *reinterpret_cast<const uint4 *>(rj + w);
            m[0] = a.x; m[1] = a.y; m[2] = a.z; m[3] = a.w;
            if (rp) {
                const uint4 x = *reinterpret_cast<const uint4 *>(rp + w);
                m[0] ^= x.x; m[1] ^= x.y; m[2] ^= x.z; m[3] ^= x.w;
            }
            if (w == 0) m[0] &= ~1u;
        }
        const int c = __popc(m[0]) + __popc(m[1]) + __popc(m[2]) + __popc(m[3]);
        int inc = c;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        const int tot = __shfl_sync(FULL, inc, 31);
        if (idx) {
            uint32_t pos = base + (uint32_t)(inc - c);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                uint32_t mk = m[k];
                while (mk) {
                    const int b = __ffs(mk) - 1;
                    mk &= mk - 1;
                    idx[pos++] = (uint32_t)((w + k) * 32 + b) - 1u;
                }
            }
        }
        base += (uint32_t)tot;
        cnt += (uint32_t)tot;
    }
    if (!idx && lane == 0) count[j] = cnt;
}

// Parent choice: for row j, the earlier row (within a look-back window)
// whose symbol set is closest in Hamming distance, if closer than empty.
__global__ void k_parent(const uint32_t *__restrict__ A, int64_t apitch, int64_t nrows,
                         const uint32_t *__restrict__ nnz, const uint32_t *__restrict__ off,
                         const uint32_t *__restrict__ idx, int lookback, int32_t *parent,
                         uint32_t *dnnz)
{
    const int64_t j = blockIdx.x;
    if (j >= nrows) return;
    __shared__ int s_best[32], s_arg[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const uint32_t nj = nnz[j];
    int best = (int)nj, arg = -1;
    const int64_t i0 = j - lookback > 0 ? j - lookback : 0;
    const uint32_t *rj = A + (size_t)j * apitch;
    for (int64_t i = i0 + threadIdx.x; i < j; i += blockDim.x) {
        // overlap of the two supports, counted from the shorter one (reading
        // the other row's bits)
        const uint32_t ni = nnz[i];
        const bool from_i = ni < nj;
        const uint32_t *ro = from_i ? rj : A + (size_t)i * apitch;
        const uint32_t kb = from_i ? off[i] : off[j], ke = from_i ? off[i + 1] : off[j + 1];
        int ov = 0;
        for (uint32_t k = kb; k < ke; k++) {
            const uint32_t s = idx[k] + 1u;
            ov += (ro[s >> 5] >> (s & 31)) & 1u;
        }
        const int d = (int)ni + (int)nj - 2 * ov;
        if (d < best || (d == best && arg >= 0 && i > arg)) { best = d; arg = (int)i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const int b2 = __shfl_xor_sync(FULL, best, o), a2 = __shfl_xor_sync(FULL, arg, o);
        if (b2 < best || (b2 == best && a2 > arg)) { best = b2; arg = a2; }
    }
    if (lane == 0) { s_best[warp] = best; s_arg[warp] = arg; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; w++)
            if (s_best[w] < best || (s_best[w] == best && s_arg[w] > arg)) { best = s_best[w]; arg = s_arg[w]; }
        if (arg >= 0 && best >= (int)nj) arg = -1;
        parent[j] = arg;
        dnnz[j] = arg >= 0 ? (uint32_t)best : nj;
    }
}

__global__ void k_cflag(const uint32_t *A, int64_t apitch, int64_t nrows, const int32_t *parent,
                        uint8_t *cflag, uint8_t *cst)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nrows) return;
    const uint32_t c = A[(size_t)j * apitch] & 1u;
    const int32_t p = parent[j];
    const uint32_t cp = p >= 0 ? (A[(size_t)p * apitch] & 1u) : 0u;
    cflag[j] = (uint8_t)(c ^ cp);
    cst[j] = (uint8_t)c;
}

// Expectation incidence: bit c of row j set when channel c's symbols meet row j.
__global__ void k_incidence(const uint32_t *__restrict__ A, int64_t apitch, int64_t row0, int64_t ntgt,
                            const uint32_t *__restrict__ sym0, const uint8_t *__restrict__ kind,
                            int64_t nch, uint32_t *inc, int64_t incPitch)
{
    const int64_t j = blockIdx.x;
    const int64_t c = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    bool hit = false;
    if (j < ntgt && c < nch) {
        const uint32_t *row = A + (size_t)(row0 + j) * apitch;
        const int k = kind[c] == CK_DEP2 ? 4 : (kind[c] == CK_DEP1 ? 2 : 1);
        for (int i = 0; i < k; i++) {
            const uint32_t s = sym0[c] + (uint32_t)i;
            hit |= ((row[s >> 5] >> (s & 31)) & 1u) != 0;
        }
    }
    const uint32_t bal = __ballot_sync(FULL, hit);
    if (j < ntgt && (threadIdx.x & 31) == 0 && c / 32 < incPitch) inc[(size_t)j * incPitch + c / 32] = bal;
}

__global__ void k_transpose_bits(const uint32_t *__restrict__ in, int64_t inPitch, int64_t nrows,
                                 int64_t ncols, uint32_t *out, int64_t outPitch)
{
    // out[c][r/32] bit r%32 = in[r][c/32] bit c%32; one warp per 32x32 block
    const int lane = threadIdx.x & 31;
    const int64_t bc = blockIdx.x, br = blockIdx.y;
    const int64_t r = br * 32 + lane;
    uint32_t x = (r < nrows && bc < inPitch) ? in[(size_t)r * inPitch + bc] : 0u;
    // 32x32 bit transpose across the warp
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
    int k = 0;
    for (int s = 16; s >= 1; s >>= 1, k++) {
        const uint32_t m = masks[k];
        const uint32_t y = __shfl_xor_sync(FULL, x, s);
        x = (lane & s) ? ((x & ~m) | ((y >> s) & m)) : ((x & m) | ((y & m) << s));
    }
    const int64_t c = bc * 32 + lane;
    if (c < ncols && br < outPitch) out[(size_t)c * outPitch + br] = x;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
// Threshold of a channel with probability p: a 32-bit draw u fires when
// u < T, T = floor(p * 2^32) clamped to 2^32 - 1.
uint32_t threshold_of(double p)
{
    if (!(p > 0.0)) return 0u;
    const double t = floor(p * 4294967296.0);
    return t >= 4294967295.0 ? 4294967295u : (uint32_t)t;
}

namespace {

struct Flat {
    std::vector<Inst> insts;
    std::vector<double> noise_p;   // probability of each noise instruction, in order (one per channel)
    std::vector<uint32_t> det_off{0}, det_refs;
    std::vector<std::vector<uint32_t>> obs;
    int64_t nmeas = 0;
    int64_t cap_sym = 0;
    int64_t nmeasfam = 0;
    int64_t nff = 0;         // feed-forward instructions
};

sp_status flatten(const sp_circuit_desc *d, Flat &F)
{
    const uint32_t n = d->num_qubits;
    for (uint32_t i = 0; i < d->num_ops; i++) {
        const sp_op &op = d->ops[i];
        const uint32_t k = op.ntargets;
        if (k && !op.targets) return set_error(SP_ERR_INVALID_ARG, "op " + std::to_string(i) + ": NULL targets");
        const uint32_t c = op.opcode;
        if (c > SP_OP_Z_IF) return set_error(SP_ERR_UNSUPPORTED_OP, "op " + std::to_string(i) + ": unknown opcode " + std::to_string(c));
        if (c <= SP_OP_DEPOLARIZE2) {
            for (uint32_t j = 0; j < k; j++)
                if (op.targets[j] >= n)
                    return set_error(SP_ERR_INVALID_ARG, "op " + std::to_string(i) + ": qubit " + std::to_string(op.targets[j]) + " >= num_qubits");
        }
        if ((c == SP_OP_CX || c == SP_OP_DEPOLARIZE2) && (k % 2))
            return set_error(SP_ERR_INVALID_ARG, "op " + std::to_string(i) + ": odd number of pair targets");
        if (c >= SP_OP_X_ERROR && c <= SP_OP_DEPOLARIZE2 && !(op.arg >= 0.0 && op.arg <= 1.0))
            return set_error(SP_ERR_INVALID_ARG, "op " + std::to_string(i) + ": probability outside [0,1]");
        const uint32_t T = threshold_of(op.arg);
        const float pf = (float)op.arg;
        uint32_t pbits;
        memcpy(&pbits, &pf, 4);
        switch (c) {
        case SP_OP_H: case SP_OP_S: case SP_OP_X: case SP_OP_Y: case SP_OP_Z: {
            const uint32_t code = c == SP_OP_H ? I_H : c == SP_OP_S ? I_S : c == SP_OP_X ? I_X : c == SP_OP_Y ? I_Y : I_Z;
            for (uint32_t j = 0; j < k; j++) F.insts.push_back({code, op.targets[j], 0, 0, 0});
        } break;
        case SP_OP_CX:
            for (uint32_t j = 0; j < k; j += 2) {
                if (op.targets[j] == op.targets[j + 1])
                    return set_error(SP_ERR_INVALID_ARG, "op " + std::to_string(i) + ": CX on one qubit");
                F.insts.push_back({I_CX, op.targets[j], op.targets[j + 1], 0, 0});
            }
            break;
        case SP_OP_M: case SP_OP_MR: case SP_OP_R: {
            const uint32_t code = c == SP_OP_M ? I_M : c == SP_OP_MR ? I_MR : I_R;
            for (uint32_t j = 0; j < k; j++) F.insts.push_back({code, op.targets[j], 0, 0, 0});
            if (c != SP_OP_R) F.nmeas += k;
            F.nmeasfam += k;
            F.cap_sym += k;
        } break;
        case SP_OP_X_ERROR: case SP_OP_Y_ERROR: case SP_OP_Z_ERROR: case SP_OP_DEPOLARIZE1: {
            const uint32_t code = c == SP_OP_X_ERROR ? I_XERR : c == SP_OP_Y_ERROR ? I_YERR : c == SP_OP_Z_ERROR ? I_ZERR : I_DEP1;
            for (uint32_t j = 0; j < k; j++) {
                F.insts.push_back({code, op.targets[j], 0, T, pbits});
                F.noise_p.push_back(op.arg);
            }
            F.cap_sym += (int64_t)k * (c == SP_OP_DEPOLARIZE1 ? 2 : 1);
        } break;
        case SP_OP_DEPOLARIZE2:
            for (uint32_t j = 0; j < k; j += 2) {
                if (op.targets[j] == op.targets[j + 1])
                    return set_error(SP_ERR_INVALID_ARG, "op " + std::to_string(i) + ": DEPOLARIZE2 on one qubit");
                F.insts.push_back({I_DEP2, op.targets[j], op.targets[j + 1], T, pbits});
                F.noise_p.push_back(op.arg);
            }
            F.cap_sym += 2 * (int64_t)k;
            break;
        case SP_OP_DETECTOR: case SP_OP_OBSERVABLE_INCLUDE: {
            std::vector<uint32_t> *dst = nullptr;
            if (c == SP_OP_OBSERVABLE_INCLUDE) {
                if (!(op.arg >= 0.0) || op.arg > 1e6 || op.arg != floor(op.arg))
                    return set_error(SP_ERR_INVALID_ARG, "op " + std::to_string(i) + ": bad observable index");
                const size_t o = (size_t)op.arg;
                if (F.obs.size() <= o) F.obs.resize(o + 1);
                dst = &F.obs[o];
            }
            for (uint32_t j = 0; j < k; j++) {
                const uint32_t lb = op.targets[j];
                if (lb < 1 || (int64_t)lb > F.nmeas)
                    return set_error(SP_ERR_INVALID_ARG, "op " + std::to_string(i) + ": rec[-" + std::to_string(lb) + "] beyond the records so far");
                const uint32_t ref = (uint32_t)(F.nmeas - lb);
                if (dst) dst->push_back(ref); else F.det_refs.push_back(ref);
            }
            if (!dst) F.det_off.push_back((uint32_t)F.det_refs.size());
        } break;
        case SP_OP_X_IF: case SP_OP_Y_IF: case SP_OP_Z_IF: {
            if (k % 2) return set_error(SP_ERR_INVALID_ARG, "op " + std::to_string(i) + ": feed-forward takes (rec, qubit) pairs");
            const uint32_t code = c == SP_OP_X_IF ? I_XIF : c == SP_OP_Y_IF ? I_YIF : I_ZIF;
            for (uint32_t j = 0; j < k; j += 2) {
                const uint32_t lb = op.targets[j], q = op.targets[j + 1];
                if (lb < 1 || (int64_t)lb > F.nmeas)
                    return set_error(SP_ERR_INVALID_ARG, "op " + std::to_string(i) + ": rec[-" + std::to_string(lb) + "] beyond the records so far");
                if (q >= n)
                    return set_error(SP_ERR_INVALID_ARG, "op " + std::to_string(i) + ": qubit " + std::to_string(q) + " >= num_qubits");
                F.insts.push_back({code, q, (uint32_t)(F.nmeas - lb), 0, 0});
                F.nff++;
            }
        } break;
        default: break;
        }
    }
    return SP_OK;
}

// The traversal's schedule.  Between two barrier ops (measurements, resets,
// feed-forward) gates and noise injections are grouped by level: an op's
// level is one more than the last level on any of its qubits, so the ops of
// one level act on disjoint qubits and commute.  Groups run in level order,
// each op of a group in parallel; barrier ops run alone, in circuit order.
// Noise ops get their index among noise ops (gi) and the number of fault
// symbols before them (sym_base): with the random outcomes so far these fix
// their symbol, channel and log slot in circuit order.
void schedule(std::vector<Inst> &insts, int n, std::vector<uint32_t> &sched, std::vector<TravStep> &steps,
              uint32_t &ninj, uint32_t &nfsym)
{
    std::vector<uint32_t> last((size_t)std::max(n, 1), 0), epoch((size_t)std::max(n, 1), 0xffffffffu);
    std::vector<std::pair<uint32_t, uint32_t>> pend;   // (level, op)
    uint32_t seg = 0;
    ninj = 0;
    nfsym = 0;
    auto flush = [&]() {
        std::stable_sort(pend.begin(), pend.end(),
                         [](const std::pair<uint32_t, uint32_t> &x, const std::pair<uint32_t, uint32_t> &y) {
                             return x.first < y.first;
                         });
        for (size_t i = 0; i < pend.size();) {
            size_t j = i;
            const uint32_t begin = (uint32_t)sched.size();
            while (j < pend.size() && pend[j].first == pend[i].first) sched.push_back(pend[j++].second);
            steps.push_back({begin, (uint32_t)sched.size(), 0u, 0u, 0u, {0u, 0u, 0u}});
            i = j;
        }
        pend.clear();
        seg++;
    };
    for (uint32_t i = 0; i < (uint32_t)insts.size(); i++) {
        Inst &in = insts[i];
        const uint32_t c = in.code;
        if (c == I_M || c == I_MR || c == I_R || c >= I_XIF) {
            flush();
            sched.push_back(i);
            steps.push_back({(uint32_t)sched.size() - 1, (uint32_t)sched.size(), 1u, ninj, nfsym, {0u, 0u, 0u}});
            continue;
        }
        if (c >= I_XERR) {
            in.gi = ninj++;
            in.sym_base = nfsym;
            nfsym += c == I_DEP2 ? 4 : (c == I_DEP1 ? 2 : 1);
        }
        const bool two = c == I_CX || c == I_DEP2;
        uint32_t lvl = 0;
        if (epoch[in.a] == seg) lvl = last[in.a];
        if (two && epoch[in.b] == seg) lvl = std::max(lvl, last[in.b]);
        lvl++;
        last[in.a] = lvl;
        epoch[in.a] = seg;
        if (two) {
            last[in.b] = lvl;
            epoch[in.b] = seg;
        }
        pend.push_back({lvl, i});
    }
    flush();
}

template <typename T>
sp_status dalloc(T **p, size_t count)
{
    if (count == 0) count = 1;
    cudaError_t e = dev_alloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_error(SP_ERR_OOM, std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) + " bytes failed");
    }
    return SP_OK;
}

struct Temp {
    std::vector<void *> ptrs;
    ~Temp() { for (void *p : ptrs) dev_free(p); }
    template <typename T> sp_status alloc(T **p, size_t count)
    {
        sp_status st = dalloc(p, count);
        if (st == SP_OK) ptrs.push_back(*p);
        return st;
    }
};

}  // namespace

sp_status build_program(const sp_circuit_desc *desc, cudaStream_t stream, sp_program *P)
{
    const auto t0 = std::chrono::steady_clock::now();
    if (desc->num_qubits > 1024)
        return set_error(SP_ERR_TOO_LARGE, "num_qubits " + std::to_string(desc->num_qubits) + " > 1024");
    if (desc->num_ops && !desc->ops) return set_error(SP_ERR_INVALID_ARG, "ops is NULL");
    Flat F;
    SP_TRY(flatten(desc, F));
    const int n = (int)desc->num_qubits;
    SP_CUDA(cudaGetDevice(&P->device));
    P->n = (uint32_t)n;
    P->n_meas = F.nmeas;
    P->n_det = (int64_t)F.det_off.size() - 1;
    P->n_obs = (int64_t)F.obs.size();
    P->n_rows = P->n_meas + P->n_det + P->n_obs;
    P->h_fault_p = F.noise_p;

    Temp tmp;
    const int Wq = std::max(1, (n + 31) / 32);
    const int64_t cap_sym = F.cap_sym;
    std::vector<uint32_t> sched;
    std::vector<TravStep> steps;
    uint32_t ninj = 0, nfsym = 0;
    schedule(F.insts, n, sched, steps, ninj, nfsym);
    const uint64_t log_cap = 2 * (uint64_t)F.insts.size() + (uint64_t)F.nmeasfam * (2 * (uint64_t)n + 8) +
                             (uint64_t)F.nff * (2 + (uint64_t)n) + 16;

    Inst *d_insts; uint32_t *d_log, *d_inj, *d_sched; uint64_t *d_logpos; uint8_t *d_symrand, *d_recconst;
    TravStep *d_steps;
    uint64_t *d_evpos;
    TraverseCounts *d_counts; uint32_t *d_gtab = nullptr;
    SP_TRY(tmp.alloc(&d_insts, F.insts.size()));
    SP_TRY(tmp.alloc(&d_sched, sched.size()));
    SP_TRY(tmp.alloc(&d_steps, steps.size()));
    uint64_t ev_cap = 1;   // a barrier op logs at most two events (a measurement and its reset)
    for (const TravStep &st : steps) ev_cap += st.barrier ? 2 : 0;
    SP_TRY(tmp.alloc(&d_evpos, ev_cap));
    SP_TRY(tmp.alloc(&d_log, log_cap));
    SP_TRY(tmp.alloc(&d_inj, (size_t)(cap_sym + 2) * Wq));
    SP_TRY(tmp.alloc(&d_logpos, (size_t)cap_sym + 2));
    SP_TRY(tmp.alloc(&d_symrand, (size_t)cap_sym + 2));
    SP_TRY(tmp.alloc(&d_recconst, (size_t)F.nmeas + 1));
    SP_TRY(tmp.alloc(&d_counts, 1));
    SP_TRY(dalloc(&P->d_chT, (size_t)cap_sym + 1));
    SP_TRY(dalloc(&P->d_chKind, (size_t)cap_sym + 1));
    SP_TRY(dalloc(&P->d_chSym0, (size_t)cap_sym + 1));
    SP_TRY(dalloc(&P->d_chP, (size_t)cap_sym + 1));
    if (!F.insts.empty()) {
        SP_CUDA(cudaMemcpyAsync(d_insts, F.insts.data(), F.insts.size() * sizeof(Inst), cudaMemcpyHostToDevice, stream));
        SP_CUDA(cudaMemcpyAsync(d_sched, sched.data(), sched.size() * 4, cudaMemcpyHostToDevice, stream));
        SP_CUDA(cudaMemcpyAsync(d_steps, steps.data(), steps.size() * sizeof(TravStep), cudaMemcpyHostToDevice, stream));
    }
    SP_CUDA(cudaMemsetAsync(d_counts, 0, sizeof(TraverseCounts), stream));
    SP_CUDA(cudaMemsetAsync(d_recconst, 0, (size_t)F.nmeas + 1, stream));

    // The tableau (4 bit-vectors of n rows per qubit, plus a pad word) lives
    // in shared memory: one CTA's when it fits next to the kernel's static
    // shared memory, else spread over a cluster of 8 CTAs (gate levels and
    // random-outcome rowsums split over the CTAs' columns: measured no slower
    // than the smallest cluster that fits at 600 qubits, 21 % faster at 800
    // and 8 % at 1,000); global memory with one CTA if no cluster can be
    // launched.
    const size_t qbytes = (4 * (size_t)Wq + 1) * 4;
    const size_t smem_cap = 192 * 1024;
    int CL = 1, qp = std::max(n, 1);
    if ((size_t)qp * qbytes > smem_cap) {
        CL = 0;
        const int q = (n + 7) / 8;
        if ((size_t)q * qbytes <= smem_cap) { CL = 8; qp = q; }
    }
    TravParams tp;
    tp.insts = d_insts; tp.sched = d_sched; tp.steps = d_steps; tp.nsteps = (int64_t)steps.size();
    tp.ninj_total = ninj; tp.nfsym_total = nfsym; tp.n = n; tp.SW = Wq;
    tp.gtab = nullptr; tp.tab_in_smem = 1; tp.log = d_log; tp.log_cap = log_cap;
    tp.inj = d_inj; tp.sym_logpos = d_logpos; tp.sym_random = d_symrand;
    tp.chT = P->d_chT; tp.chKind = P->d_chKind; tp.chSym0 = P->d_chSym0; tp.chP = P->d_chP;
    tp.rec_const = d_recconst; tp.counts = d_counts; tp.ev_pos = d_evpos; tp.ev_cap = ev_cap;
    tp.qp = qp;
    bool launched = false;
    // SP_TRAVERSE_NO_CLUSTER set: the one-CTA fallback (tableau in global
    // memory) even where a cluster could be launched -- for testing that path
    if (CL > 1 && !getenv("SP_TRAVERSE_NO_CLUSTER")) {
        const size_t smem = (size_t)qp * qbytes;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)CL);
        cfg.blockDim = dim3(TRAV_THREADS);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t e = cudaSuccess;
        SP_CUDA(max_dynamic_smem(k_traverse<8>));
        e = cudaLaunchKernelEx(&cfg, k_traverse<8>, tp);
        if (e == cudaSuccess) launched = true;
        else cudaGetLastError();
    }
    if (!launched) {
        const bool in_smem = CL == 1;
        if (!in_smem) SP_TRY(tmp.alloc(&d_gtab, (size_t)std::max(n, 1) * (4 * (size_t)Wq + 1)));
        tp.gtab = d_gtab;
        tp.tab_in_smem = in_smem ? 1 : 0;
        tp.qp = std::max(n, 1);
        SP_CUDA(max_dynamic_smem(k_traverse<1>));
        k_traverse<1><<<1, TRAV_THREADS, in_smem ? (size_t)std::max(n, 1) * qbytes : 0, stream>>>(tp);
    }
    SP_CUDA(cudaGetLastError());
    TraverseCounts hc;
    SP_CUDA(cudaMemcpyAsync(&hc, d_counts, sizeof hc, cudaMemcpyDeviceToHost, stream));
    SP_CUDA(cudaStreamSynchronize(stream));
    if (hc.err == 1) return set_error(SP_ERR_TOO_LARGE, "traversal log overflow");
    if (hc.err == 2) return set_error(SP_ERR_CUDA, "traversal self-check failed: odd product phase");
    if ((int64_t)hc.nrec != F.nmeas) return set_error(SP_ERR_CUDA, "traversal record count mismatch");
    P->n_sym = hc.nsym;
    P->n_ch = hc.nch;
    P->log_len = (int64_t)hc.log_len;

    // ---- K2: replay every symbol column ---------------------------------
    P->apitch = ceil_div(P->n_sym + 1, 32);
    P->apitch = ceil_div(P->apitch, 4) * 4;
    const size_t arows = (size_t)std::max<int64_t>(P->n_rows, 1);
    SP_TRY(dalloc(&P->d_A, arows * P->apitch));
    SP_CUDA(cudaMemsetAsync(P->d_A, 0, arows * P->apitch * 4, stream));
    if (P->n_sym > 0 && n > 0) {
        const int64_t nblk = ceil_div(P->n_sym + 1, 1024);
        // eight warps share a CTA's table where row lists are long enough to
        // split; one warp otherwise
        if (n >= REPLAY_SPLIT_MIN_N) {
            const size_t vsm = ((size_t)n + 8) * 32 * 4;
            SP_CUDA(max_dynamic_smem(k_replay<8>));
            k_replay<8><<<(unsigned)nblk, 256, vsm, stream>>>(d_log, hc.log_len, d_evpos, hc.nev, d_inj, Wq, d_logpos,
                                                               d_symrand, hc.nsym, n, P->d_A, P->apitch);
        } else {
            const size_t vsm = ((size_t)n + 1) * 32 * 4;
            SP_CUDA(max_dynamic_smem(k_replay<1>));
            k_replay<1><<<(unsigned)nblk, 32, vsm, stream>>>(d_log, hc.log_len, d_evpos, hc.nev, d_inj, Wq, d_logpos,
                                                              d_symrand, hc.nsym, n, P->d_A, P->apitch);
        }
        SP_CUDA(cudaGetLastError());
    }
    if (P->n_meas > 0) {
        k_merge_const<<<(unsigned)ceil_div(P->n_meas, 256), 256, 0, stream>>>(P->d_A, P->apitch, d_recconst, P->n_meas);
        SP_CUDA(cudaGetLastError());
    }
    // ---- K3: detector and observable rows -----------------------------------
    std::vector<uint32_t> xoff(F.det_off), xrefs(F.det_refs);
    for (auto &o : F.obs) {
        xrefs.insert(xrefs.end(), o.begin(), o.end());
        xoff.push_back((uint32_t)xrefs.size());
    }
    P->h_xoff = xoff;
    P->h_xrefs = xrefs;
    const int64_t ntgt = P->n_det + P->n_obs;
    if (ntgt > 0) {
        uint32_t *d_xoff, *d_xrefs;
        SP_TRY(tmp.alloc(&d_xoff, xoff.size()));
        SP_TRY(tmp.alloc(&d_xrefs, std::max<size_t>(xrefs.size(), 1)));
        SP_CUDA(cudaMemcpyAsync(d_xoff, xoff.data(), xoff.size() * 4, cudaMemcpyHostToDevice, stream));
        if (!xrefs.empty())
            SP_CUDA(cudaMemcpyAsync(d_xrefs, xrefs.data(), xrefs.size() * 4, cudaMemcpyHostToDevice, stream));
        k_xor_rows<<<(unsigned)ntgt, 128, 0, stream>>>(P->d_A, P->apitch, d_xoff, d_xrefs, ntgt, P->n_meas);
        SP_CUDA(cudaGetLastError());
    }
    SP_TRY(finish_program(P, stream));
    P->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return SP_OK;
}

// Everything the sampler and the expectations derive from the coefficient
// rows (P->d_A) and the channel table: run after the traversal by
// build_program and after the rows are restored by sp_load.
sp_status finish_program(sp_program *P, cudaStream_t stream)
{
    Temp tmp;
    const int64_t ntgt = P->n_det + P->n_obs;
    // number of random symbols
    {
        std::vector<uint8_t> hk((size_t)P->n_ch);
        std::vector<uint32_t> hs((size_t)P->n_ch);
        if (P->n_ch) {
            SP_CUDA(cudaMemcpy(hk.data(), P->d_chKind, (size_t)P->n_ch, cudaMemcpyDeviceToHost));
            SP_CUDA(cudaMemcpy(hs.data(), P->d_chSym0, (size_t)P->n_ch * 4, cudaMemcpyDeviceToHost));
        }
        P->n_rand = std::count(hk.begin(), hk.end(), (uint8_t)CK_RANDOM);
        // a detector or observable with a random-measurement symbol is rejected
        if (ntgt > 0 && P->n_rand > 0) {
            std::vector<uint32_t> mask((size_t)P->apitch, 0u);
            for (int64_t c = 0; c < P->n_ch; c++)
                if (hk[c] == CK_RANDOM) mask[hs[c] >> 5] |= 1u << (hs[c] & 31);
            uint32_t *d_mask; int *d_bad;
            SP_TRY(tmp.alloc(&d_mask, (size_t)P->apitch));
            SP_TRY(tmp.alloc(&d_bad, 1));
            const int big = 0x7fffffff;
            SP_CUDA(cudaMemcpyAsync(d_mask, mask.data(), (size_t)P->apitch * 4, cudaMemcpyHostToDevice, stream));
            SP_CUDA(cudaMemcpyAsync(d_bad, &big, 4, cudaMemcpyHostToDevice, stream));
            k_check_random<<<(unsigned)ntgt, 128, 0, stream>>>(P->d_A, P->apitch, P->n_meas, ntgt, d_mask, d_bad);
            SP_CUDA(cudaGetLastError());
            int bad;
            SP_CUDA(cudaMemcpyAsync(&bad, d_bad, 4, cudaMemcpyDeviceToHost, stream));
            SP_CUDA(cudaStreamSynchronize(stream));
            if (bad != big) {
                std::string what = bad < P->n_det ? "detector " + std::to_string(bad)
                                                  : "observable " + std::to_string(bad - P->n_det);
                return set_error(SP_ERR_NONDETERMINISTIC_DETECTOR, what + " depends on a random measurement outcome");
            }
        }
        std::vector<float> kap((size_t)std::max<int64_t>(P->n_ch, 1), 0.f);
        for (int64_t c = 0; c < P->n_ch; c++)
            kap[c] = hk[c] == CK_DEP1 ? 2.0f / 3.0f : hk[c] == CK_DEP2 ? 8.0f / 15.0f : hk[c] == CK_BERN ? 1.0f : 0.0f;
        SP_TRY(dalloc(&P->d_kappa, kap.size()));
        SP_CUDA(cudaMemcpy(P->d_kappa, kap.data(), kap.size() * 4, cudaMemcpyHostToDevice));
    }
    // ---- sampler program: full-row support, parent choice, delta rows ----
    const int64_t R = P->n_rows;
    SP_TRY(dalloc(&P->d_parent, (size_t)std::max<int64_t>(R, 1)));
    SP_TRY(dalloc(&P->d_cflag, (size_t)std::max<int64_t>(R, 1)));
    SP_TRY(dalloc(&P->d_const, (size_t)std::max<int64_t>(R, 1)));
    SP_TRY(dalloc(&P->d_rowOff, (size_t)R + 1));
    if (R > 0) {
        uint32_t *d_cnt, *d_off, *d_fidx, *d_dnnz;
        SP_TRY(tmp.alloc(&d_cnt, (size_t)R));
        SP_TRY(tmp.alloc(&d_off, (size_t)R + 1));
        SP_TRY(tmp.alloc(&d_dnnz, (size_t)R));
        const unsigned rb = (unsigned)ceil_div(R, 8);
        k_row_csr<<<rb, 256, 0, stream>>>(P->d_A, P->apitch, R, nullptr, d_cnt, nullptr, nullptr);
        SP_CUDA(cudaGetLastError());
        std::vector<uint32_t> cnt((size_t)R), off((size_t)R + 1, 0);
        SP_CUDA(cudaMemcpyAsync(cnt.data(), d_cnt, (size_t)R * 4, cudaMemcpyDeviceToHost, stream));
        SP_CUDA(cudaStreamSynchronize(stream));
        uint64_t tot = 0;
        for (int64_t j = 0; j < R; j++) { off[j] = (uint32_t)tot; tot += cnt[j]; }
        off[R] = (uint32_t)tot;
        if (tot >= 0xffffffffull) return set_error(SP_ERR_TOO_LARGE, "more than 2^32 nonzero coefficients");
        P->nnz_rows = (int64_t)tot;
        // the full rows stay with the program where they are small: the
        // staged product gathers them row-parallel when few shots leave the
        // parent chains too little parallelism
        if (tot <= FULL_ROWS_KEEP) {
            SP_TRY(dalloc(&P->d_fullIdx, (size_t)std::max<uint64_t>(tot, 1)));
            SP_TRY(dalloc(&P->d_fullOff, (size_t)R + 1));
            d_fidx = P->d_fullIdx;
            SP_CUDA(cudaMemcpyAsync(P->d_fullOff, off.data(), ((size_t)R + 1) * 4, cudaMemcpyHostToDevice, stream));
        } else {
            SP_TRY(tmp.alloc(&d_fidx, (size_t)tot));
        }
        SP_CUDA(cudaMemcpyAsync(d_off, off.data(), ((size_t)R + 1) * 4, cudaMemcpyHostToDevice, stream));
        k_row_csr<<<rb, 256, 0, stream>>>(P->d_A, P->apitch, R, nullptr, nullptr, d_off, d_fidx);
        k_parent<<<(unsigned)R, 128, 0, stream>>>(P->d_A, P->apitch, R, d_cnt, d_off, d_fidx,
                                                  PARENT_LOOKBACK, P->d_parent, d_dnnz);
        SP_CUDA(cudaGetLastError());
        std::vector<uint32_t> dn((size_t)R), doff((size_t)R + 1, 0);
        SP_CUDA(cudaMemcpyAsync(dn.data(), d_dnnz, (size_t)R * 4, cudaMemcpyDeviceToHost, stream));
        SP_CUDA(cudaStreamSynchronize(stream));
        tot = 0;
        for (int64_t j = 0; j < R; j++) { doff[j] = (uint32_t)tot; tot += dn[j]; }
        doff[R] = (uint32_t)tot;
        P->nnz_delta = (int64_t)tot;
        SP_TRY(dalloc(&P->d_idx, (size_t)tot));
        SP_CUDA(cudaMemcpyAsync(P->d_rowOff, doff.data(), ((size_t)R + 1) * 4, cudaMemcpyHostToDevice, stream));
        k_row_csr<<<rb, 256, 0, stream>>>(P->d_A, P->apitch, R, P->d_parent, nullptr, P->d_rowOff, P->d_idx);
        k_cflag<<<(unsigned)ceil_div(R, 256), 256, 0, stream>>>(P->d_A, P->apitch, R, P->d_parent, P->d_cflag, P->d_const);
        SP_CUDA(cudaGetLastError());
    } else {
        const uint32_t z = 0;
        SP_CUDA(cudaMemcpyAsync(P->d_rowOff, &z, 4, cudaMemcpyHostToDevice, stream));
    }
    // ---- expectation incidence (targets x channels) and its transpose -----
    P->incPitch = std::max<int64_t>(1, ceil_div(P->n_ch, 32));
    P->incTPitch = std::max<int64_t>(1, ceil_div(ntgt, 32));
    SP_TRY(dalloc(&P->d_inc, (size_t)std::max<int64_t>(ntgt, 1) * P->incPitch));
    SP_TRY(dalloc(&P->d_incT, (size_t)std::max<int64_t>(P->n_ch, 1) * P->incTPitch));
    SP_CUDA(cudaMemsetAsync(P->d_inc, 0, (size_t)std::max<int64_t>(ntgt, 1) * P->incPitch * 4, stream));
    SP_CUDA(cudaMemsetAsync(P->d_incT, 0, (size_t)std::max<int64_t>(P->n_ch, 1) * P->incTPitch * 4, stream));
    if (ntgt > 0 && P->n_ch > 0) {
        dim3 g((unsigned)ntgt, (unsigned)ceil_div(P->n_ch, 128));
        k_incidence<<<g, 128, 0, stream>>>(P->d_A, P->apitch, P->n_meas, ntgt, P->d_chSym0, P->d_chKind,
                                            P->n_ch, P->d_inc, P->incPitch);
        dim3 g2((unsigned)P->incPitch, (unsigned)ceil_div(ntgt, 32));
        k_transpose_bits<<<g2, 32, 0, stream>>>(P->d_inc, P->incPitch, ntgt, P->n_ch, P->d_incT, P->incTPitch);
        SP_CUDA(cudaGetLastError());
    }
    P->h_const.assign((size_t)R, 0);
    if (R > 0) SP_CUDA(cudaMemcpyAsync(P->h_const.data(), P->d_const, (size_t)R, cudaMemcpyDeviceToHost, stream));
    SP_CUDA(cudaStreamSynchronize(stream));
    const double cells = (double)std::max<int64_t>(R, 1) * (double)std::max<int64_t>(P->n_sym, 1);
    P->density = (double)P->nnz_rows / cells;
    SP_TRY(build_fused_program(P, stream));
    SP_TRY(autotune(P, stream));
    P->chunk_shots = default_chunk(P);
    SP_TRY(choose_path(P, stream));
    return SP_OK;
}

}  // namespace sp
