// sp_build.cu -- Algorithm 1 "Initialization" on the GPU (arXiv 2311.03906).
//
// The symbolic tableau of Eq. stabilizer3 is 2n x (2n + n_s + 1) bits.  By
// Fact 2 every branch of A-G's algorithm depends only on the X/Z part, so the
// traversal runs in two passes:
//   K1 k_traverse   one CTA walks the ops in order over the X/Z tableau plus
//                   the constant phase column (Init-C, Fact 1, Init-M on
//                   column 0) and writes a log of the row operations that
//                   touch symbol columns, plus each fault symbol's injection
//                   column (Init-P: X^{s} flips rows with z_a = 1, Z^{s} rows
//                   with x_a = 1);
//   K2 k_replay     every symbol column is replayed through that log from
//                   the moment its symbol appears, 32 columns per thread as
//                   bit-sliced words in shared memory.  The outcome vector of
//                   a measurement (Init-M) is the XOR of its row set.
// Only stabilizer-row phases are replayed: destabilizer phases never feed a
// stabilizer phase or an outcome in A-G's algorithm.  Detector and
// observable rows are XORs of measurement rows (K3).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "sp_internal.h"

namespace sp {

constexpr int TRAV_THREADS = 1024;
constexpr uint32_t FULL = 0xffffffffu;
constexpr int PARENT_LOOKBACK = 512;

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

__device__ __forceinline__ int warp_min(int v)
{
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

__device__ __forceinline__ int warp_sum(int v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Exclusive prefix sum of c over a 1024-thread block; *total gets the sum.
__device__ __forceinline__ int block_excl_scan(int c, int *s_warp, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = c;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int v = s_warp[lane];
        int vi = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(FULL, vi, o);
            if (lane >= o) vi += y;
        }
        s_warp[lane] = vi - v;
        if (lane == 31) s_warp[32] = vi;
    }
    __syncthreads();
    int off = s_warp[warp] + inc - c;
    *total = s_warp[32];
    __syncthreads();
    return off;
}

struct TravParams {
    const Inst *insts;
    int64_t ninst;
    int n, Wq, R2;
    uint32_t *gtab;          // used when the tableau does not fit in shared memory
    int tab_in_smem;
    uint32_t *log;
    uint64_t log_cap;
    uint32_t *inj;           // [(cap_sym + 2) * Wq]
    uint64_t *sym_logpos;    // [cap_sym + 2]
    uint8_t *sym_random;     // [cap_sym + 2]
    uint32_t *chT;
    uint8_t *chKind;
    uint32_t *chSym0;
    float *chP;
    uint8_t *rec_const;
    TraverseCounts *counts;
};

// K1: the X/Z pass.  Thread t owns tableau rows t and t + 1024; rows 0..n-1
// are stabilizers, n..2n-1 destabilizers (stabilizer i pairs with row n+i).
// Layout: X[w * R2 + row] (32 qubits per word, rows contiguous per word).
__global__ void __launch_bounds__(TRAV_THREADS, 1) k_traverse(TravParams P)
{
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int s_p, s_e, s_err;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int n = P.n, NR = 2 * n, Wq = P.Wq, R2 = P.R2;
    int *s_warp = reinterpret_cast<int *>(smem);          // 64 ints
    int *s_list = s_warp + 64;                            // 2048 ints
    uint8_t *r = reinterpret_cast<uint8_t *>(s_list + 2048); // R2 bytes (stabilizer phases)
    uint32_t *X = P.tab_in_smem ? reinterpret_cast<uint32_t *>(r + R2) : P.gtab;
    uint32_t *Z = X + (size_t)Wq * R2;
    const int row0 = t, row1 = t + TRAV_THREADS;

    for (int w = 0; w < Wq; w++) {
        for (int k = 0; k < 2; k++) {
            int row = t + k * TRAV_THREADS;
            if (row >= R2) break;
            uint32_t xv = 0, zv = 0;
            if (row < n) {
                if ((row >> 5) == w) zv = 1u << (row & 31);
            } else if (row < NR) {
                int q = row - n;
                if ((q >> 5) == w) xv = 1u << (q & 31);
            }
            X[(size_t)w * R2 + row] = xv;
            Z[(size_t)w * R2 + row] = zv;
        }
    }
    if (row0 < R2) r[row0] = 0;
    if (row1 < R2) r[row1] = 0;
    if (t == 0) s_err = 0;
    __syncthreads();

    uint32_t nsym = 0, nch = 0, nrec = 0, err = 0;
    uint64_t lp = 0;
    for (int64_t ii = 0; ii < P.ninst; ii++) {
        const Inst in = P.insts[ii];
        const uint32_t code = in.code;
        const uint32_t a = in.a, wa = a >> 5, ma = 1u << (a & 31);
        if (code <= I_Z) {
            // Init-C (H, S, CX: A-G's column updates, phase column 0) and
            // Pauli gates (Fact 1).  Rows are independent: no barrier.
            for (int k = 0; k < 2; k++) {
                const int row = t + k * TRAV_THREADS;
                if (row >= NR) break;
                uint32_t *px = X + (size_t)wa * R2 + row;
                uint32_t *pz = Z + (size_t)wa * R2 + row;
                const bool stab = row < n;
                switch (code) {
                case I_H: {
                    uint32_t xv = *px, zv = *pz, xb = xv & ma, zb = zv & ma;
                    if (stab && xb && zb) r[row] ^= 1;
                    *px = (xv & ~ma) | zb;
                    *pz = (zv & ~ma) | xb;
                } break;
                case I_S: {
                    uint32_t xv = *px, zv = *pz;
                    if (stab && (xv & ma) && (zv & ma)) r[row] ^= 1;
                    *pz = zv ^ (xv & ma);
                } break;
                case I_X: if (stab && (*pz & ma)) r[row] ^= 1; break;
                case I_Z: if (stab && (*px & ma)) r[row] ^= 1; break;
                case I_Y: if (stab && ((*px ^ *pz) & ma)) r[row] ^= 1; break;
                case I_CX: {
                    const uint32_t b = in.b, wb = b >> 5, mb = 1u << (b & 31);
                    uint32_t *qx = X + (size_t)wb * R2 + row;
                    uint32_t *qz = Z + (size_t)wb * R2 + row;
                    const bool xa = (*px & ma) != 0, za = (*pz & ma) != 0;
                    const bool xb = (*qx & mb) != 0, zb = (*qz & mb) != 0;
                    if (stab && xa && zb && (xb == za)) r[row] ^= 1;
                    if (xa) *qx ^= mb;
                    if (zb) *pz ^= ma;
                } break;
                default: break;
                }
            }
            continue;
        }
        if (code >= I_XIF) {
            // Feed-forward (the conditional Paulis of Sec. 6): P^e on qubit a
            // with e the form of record in.b.  A stabilizer row that
            // anticommutes with P (X: z_a, Z: x_a, Y: x_a ^ z_a) gets e: its
            // constant bit here, its symbol part in the replay (EV_FF).
            if (lp + 2 + (uint64_t)n > P.log_cap) { err = 1; break; }
            const bool useZ = code != I_ZIF, useX = code != I_XIF;
            __syncthreads();   // the record's constant was written by thread 0
            const uint32_t e_const = P.rec_const[in.b];
            int f = 0;
            if (t < n) {
                const bool zb = (Z[(size_t)wa * R2 + t] & ma) != 0, xb = (X[(size_t)wa * R2 + t] & ma) != 0;
                f = ((useZ && zb) != (useX && xb)) ? 1 : 0;
            }
            int total;
            const int off = block_excl_scan(f, s_warp, &total);
            if (f) {
                P.log[lp + 2 + off] = (uint32_t)t;
                if (e_const) r[t] ^= 1;
            }
            if (t == 0) {
                P.log[lp] = (EV_FF << 24) | (uint32_t)total;
                P.log[lp + 1] = in.b;
            }
            lp += 2 + (uint64_t)total;
            continue;
        }
        if (code >= I_XERR) {
            // Init-P: record each symbol's injection column over the
            // stabilizer rows (X-type part: z_q, Z-type part: x_q).
            const int k = (code == I_DEP2) ? 4 : (code == I_DEP1 ? 2 : 1);
            if (lp + 2 > P.log_cap) { err = 1; break; }
            const uint32_t s0 = nsym + 1;
            for (int j = 0; j < k; j++) {
                const uint32_t q = (j < 2) ? a : in.b;
                int useZ, useX;
                if (code == I_XERR) { useZ = 1; useX = 0; }
                else if (code == I_ZERR) { useZ = 0; useX = 1; }
                else if (code == I_YERR) { useZ = 1; useX = 1; }
                else { useZ = !(j & 1); useX = j & 1; }
                uint32_t bit = 0;
                if (t < n) {
                    const uint32_t w = q >> 5, m = 1u << (q & 31);
                    const uint32_t xb = (X[(size_t)w * R2 + t] & m) ? 1u : 0u;
                    const uint32_t zb = (Z[(size_t)w * R2 + t] & m) ? 1u : 0u;
                    bit = (useZ & zb) ^ (useX & xb);
                }
                const uint32_t bal = __ballot_sync(FULL, bit);
                if (lane == 0 && warp < Wq) P.inj[(size_t)(s0 + j) * Wq + warp] = bal;
            }
            if (t == 0) {
                P.chT[nch] = in.aux;
                P.chP[nch] = __uint_as_float(in.pbits);
                P.chKind[nch] = (k == 1) ? CK_BERN : (k == 2 ? CK_DEP1 : CK_DEP2);
                P.chSym0[nch] = s0;
                P.log[lp] = (EV_INJECT << 24) | (uint32_t)k;
                P.log[lp + 1] = s0;
                for (int j = 0; j < k; j++) { P.sym_logpos[s0 + j] = lp; P.sym_random[s0 + j] = 0; }
            }
            lp += 2;
            nsym += k;
            nch++;
            continue;
        }
        // ---- Init-M (M, MR, R) ------------------------------------------
        const bool recorded = (code != I_R), reset = (code != I_M);
        if (lp + 2 * (uint64_t)n + 8 > P.log_cap) { err = 1; break; }
        __syncthreads();
        int cand = (t < n && (X[(size_t)wa * R2 + t] & ma)) ? t : 0x7fffffff;
        cand = warp_min(cand);
        if (lane == 0) s_warp[warp] = cand;
        __syncthreads();
        if (warp == 0) {
            int v = warp_min(s_warp[lane]);
            if (lane == 0) s_p = v;
        }
        __syncthreads();
        const int p = s_p;
        const uint32_t rec = recorded ? nrec : NO_REC;
        uint32_t e_const;
        if (p != 0x7fffffff) {
            // random outcome: every other row with x_a = 1 becomes P_p * row
            const bool f0 = row0 < NR && row0 != p && (X[(size_t)wa * R2 + row0] & ma);
            const bool f1 = row1 < NR && row1 != p && (X[(size_t)wa * R2 + row1] & ma);
            const int c = (row0 < n && f0) ? 1 : 0;
            int total;
            const int off = block_excl_scan(c, s_warp, &total);
            if (c) P.log[lp + 4 + off] = (uint32_t)row0;
            for (int k = 0; k < 2; k++) {
                const bool f = k ? f1 : f0;
                if (!f) continue;
                const int row = k ? row1 : row0;
                int g = 0;
                for (int w = 0; w < Wq; w++) {
                    const uint32_t xp = X[(size_t)w * R2 + p], zp = Z[(size_t)w * R2 + p];
                    const uint32_t xr = X[(size_t)w * R2 + row], zr = Z[(size_t)w * R2 + row];
                    if (row < n) g += gcount(xp, zp, xr, zr);
                    X[(size_t)w * R2 + row] = xr ^ xp;
                    Z[(size_t)w * R2 + row] = zr ^ zp;
                }
                if (row < n) r[row] = (uint8_t)((((2 * r[row] + 2 * r[p] + g) & 3) == 2) ? 1 : 0);
            }
            __syncthreads();
            const uint32_t s = nsym + 1;
            if (t == 0) {
                for (int w = 0; w < Wq; w++) {
                    X[(size_t)w * R2 + n + p] = X[(size_t)w * R2 + p];
                    Z[(size_t)w * R2 + n + p] = Z[(size_t)w * R2 + p];
                    X[(size_t)w * R2 + p] = 0;
                    Z[(size_t)w * R2 + p] = ((uint32_t)w == wa) ? ma : 0u;
                }
                r[p] = 0;
                P.log[lp] = (EV_MRAND << 24) | (uint32_t)total;
                P.log[lp + 1] = (uint32_t)p;
                P.log[lp + 2] = s;
                P.log[lp + 3] = rec;
                P.chT[nch] = 0x80000000u;
                P.chP[nch] = 0.5f;
                P.chKind[nch] = CK_RANDOM;
                P.chSym0[nch] = s;
                P.sym_logpos[s] = lp;
                P.sym_random[s] = 1;
            }
            lp += 4 + (uint64_t)total;
            nsym++;
            nch++;
            e_const = 0;
            __syncthreads();
        } else {
            // deterministic outcome: product of the stabilizers paired with
            // destabilizers that have x_a = 1
            const bool f0 = row0 >= n && row0 < NR && (X[(size_t)wa * R2 + row0] & ma);
            const bool f1 = row1 < NR && (X[(size_t)wa * R2 + row1] & ma);
            const int c = (int)f0 + (int)f1;
            int total;
            int off = block_excl_scan(c, s_warp, &total);
            if (f0) { s_list[off] = row0 - n; P.log[lp + 2 + off] = (uint32_t)(row0 - n); off++; }
            if (f1) { s_list[off] = row1 - n; P.log[lp + 2 + off] = (uint32_t)(row1 - n); }
            __syncthreads();
            if (warp == 0) {
                uint32_t ax = 0, az = 0;
                int g = 0, rs = 0;
                for (int j = 0; j < total; j++) {
                    const int i = s_list[j];
                    if (lane < Wq) {
                        const uint32_t xi = X[(size_t)lane * R2 + i], zi = Z[(size_t)lane * R2 + i];
                        g += gcount(xi, zi, ax, az);
                        ax ^= xi;
                        az ^= zi;
                    }
                    if (lane == 0) rs += r[i];
                }
                g = warp_sum(g);
                if (lane == 0) {
                    const int tot = (2 * rs + g) & 3;
                    s_e = (tot == 2) ? 1 : 0;
                    if (tot & 1) s_err = 2;
                }
            }
            if (t == 0) {
                P.log[lp] = (EV_MDET << 24) | (uint32_t)total;
                P.log[lp + 1] = rec;
            }
            lp += 2 + (uint64_t)total;
            __syncthreads();
            e_const = (uint32_t)s_e;
        }
        if (recorded) {
            if (t == 0) P.rec_const[nrec] = (uint8_t)e_const;
            nrec++;
        }
        if (reset) {
            // conditional X^e on qubit a: flip every stabilizer with z_a = 1
            const int f = (t < n && (Z[(size_t)wa * R2 + t] & ma)) ? 1 : 0;
            int total;
            const int off = block_excl_scan(f, s_warp, &total);
            if (f) {
                P.log[lp + 1 + off] = (uint32_t)t;
                if (e_const) r[t] ^= 1;
            }
            if (t == 0) P.log[lp] = (EV_RESET << 24) | (uint32_t)total;
            lp += 1 + (uint64_t)total;
        }
    }
    __syncthreads();
    if (t == 0) {
        P.counts->log_len = lp;
        P.counts->nsym = nsym;
        P.counts->nch = nch;
        P.counts->nrec = nrec;
        P.counts->err = err ? err : (uint32_t)s_err;
    }
}

// K2: column-parallel replay.  One warp per CTA; lane l owns symbols
// 32*(32*blockIdx + l) .. +31 as one bit-sliced word per stabilizer row.
__global__ void __launch_bounds__(32) k_replay(const uint32_t *__restrict__ log, uint64_t log_len,
                                               const uint32_t *__restrict__ inj, int Wq,
                                               const uint64_t *__restrict__ sym_logpos, uint32_t nsym,
                                               int n, uint32_t *__restrict__ A, int64_t apitch)
{
    extern __shared__ uint32_t v[];  // [n][32]
    const int lane = threadIdx.x;
    const int64_t g = (int64_t)blockIdx.x * 32 + lane;
    uint32_t s_first = (uint32_t)blockIdx.x * 1024u;
    if (s_first == 0) s_first = 1;
    if (s_first > nsym) return;
    for (int i = 0; i < n; i++) v[i * 32 + lane] = 0;
    __syncwarp();
    const uint32_t lo = (uint32_t)g * 32u, hi = lo + 32u;
    const bool write = g < apitch;
    uint64_t pos = sym_logpos[s_first];
    uint32_t e = 0;
    while (pos < log_len) {
        const uint32_t h = log[pos];
        const uint32_t ev = h >> 24, cnt = h & 0xffffffu;
        // every event must fit in the log and name rows below n
        const uint64_t len = ev == EV_INJECT ? 2 : ev == EV_MRAND ? 4 + (uint64_t)cnt
                           : (ev == EV_MDET || ev == EV_FF) ? 2 + (uint64_t)cnt : 1 + (uint64_t)cnt;
        if (pos + len > log_len) break;
        if (ev == EV_INJECT) {
            const uint32_t s0 = log[pos + 1];
            for (uint32_t s = s0; s < s0 + cnt; s++) {
                if (s >= lo && s < hi) {
                    const uint32_t bit = 1u << (s & 31);
                    const uint32_t *col = inj + (size_t)s * Wq;
                    for (int w = 0; w < Wq; w++) {
                        uint32_t m = col[w];
                        while (m) {
                            const int b = __ffs(m) - 1;
                            m &= m - 1;
                            if (w * 32 + b < n) v[(w * 32 + b) * 32 + lane] ^= bit;
                        }
                    }
                }
            }
            pos += 2;
        } else if (ev == EV_MRAND) {
            const uint32_t p = min(log[pos + 1], (uint32_t)n - 1u), s = log[pos + 2], rec = log[pos + 3];
            const uint32_t vp = v[p * 32 + lane];
            const uint32_t *rows = log + pos + 4;
            for (uint32_t j = 0; j < cnt; j++) {
                const uint32_t i = rows[j];
                if (i < (uint32_t)n) v[i * 32 + lane] ^= vp;
            }
            e = (s >= lo && s < hi) ? (1u << (s & 31)) : 0u;
            v[p * 32 + lane] = e;
            if (rec != NO_REC && write) A[(size_t)rec * apitch + g] = e;
            pos += 4 + cnt;
        } else if (ev == EV_MDET) {
            const uint32_t rec = log[pos + 1];
            const uint32_t *rows = log + pos + 2;
            uint32_t acc0 = 0, acc1 = 0;
            uint32_t j = 0;
            for (; j + 1 < cnt; j += 2) {
                const uint32_t i0 = min(rows[j], (uint32_t)n - 1u), i1 = min(rows[j + 1], (uint32_t)n - 1u);
                acc0 ^= v[i0 * 32 + lane];
                acc1 ^= v[i1 * 32 + lane];
            }
            if (j < cnt) acc0 ^= v[min(rows[j], (uint32_t)n - 1u) * 32 + lane];
            e = acc0 ^ acc1;
            if (rec != NO_REC && write) A[(size_t)rec * apitch + g] = e;
            pos += 2 + cnt;
        } else if (ev == EV_FF) {
            // the record's symbol word for this lane: written above by this
            // same thread, or still zero if the record precedes its symbols
            const uint32_t rec = log[pos + 1];
            const uint32_t ef = write ? A[(size_t)rec * apitch + g] : 0u;
            const uint32_t *rows = log + pos + 2;
            for (uint32_t j = 0; j < cnt; j++) {
                const uint32_t i = rows[j];
                if (i < (uint32_t)n) v[i * 32 + lane] ^= ef;
            }
            pos += 2 + cnt;
        } else {
            const uint32_t *rows = log + pos + 1;
            for (uint32_t j = 0; j < cnt; j++) {
                const uint32_t i = rows[j];
                if (i < (uint32_t)n) v[i * 32 + lane] ^= e;
            }
            pos += 1 + cnt;
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

__global__ void k_random_mask(const uint8_t *sym_random, uint32_t nsym, uint32_t *mask, int64_t apitch)
{
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= apitch) return;
    uint32_t m = 0;
    for (int b = 0; b < 32; b++) {
        const int64_t s = w * 32 + b;
        if (s >= 1 && s <= (int64_t)nsym && sym_random[s]) m |= 1u << b;
    }
    mask[w] = m;
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
    for (int64_t w0 = 0; w0 < apitch; w0 += 32) {
        const int64_t w = w0 + lane;
        uint32_t m = 0;
        if (w < apitch) {
            m = rj[w];
            if (rp) m ^= rp[w];
            if (w == 0) m &= ~1u;
        }
        const int c = __popc(m);
        int inc = c;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        const int tot = __shfl_sync(FULL, inc, 31);
        if (idx) {
            uint32_t pos = base + (uint32_t)(inc - c);
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                idx[pos++] = (uint32_t)(w * 32 + b) - 1u;
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
    for (int64_t i = i0 + threadIdx.x; i < j; i += blockDim.x) {
        const uint32_t *ri = A + (size_t)i * apitch;
        int ov = 0;
        for (uint32_t k = off[j]; k < off[j + 1]; k++) {
            const uint32_t s = idx[k] + 1u;
            ov += (ri[s >> 5] >> (s & 31)) & 1u;
        }
        const int d = (int)nnz[i] + (int)nj - 2 * ov;
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
namespace {

struct Flat {
    std::vector<Inst> insts;
    std::vector<uint32_t> det_off{0}, det_refs;
    std::vector<std::vector<uint32_t>> obs;
    int64_t nmeas = 0;
    int64_t cap_sym = 0;
    int64_t nmeasfam = 0;
    int64_t nff = 0;         // feed-forward instructions
};

uint32_t threshold_of(double p)
{
    if (!(p > 0.0)) return 0u;
    const double t = floor(p * 4294967296.0);
    return t >= 4294967295.0 ? 4294967295u : (uint32_t)t;
}

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
            for (uint32_t j = 0; j < k; j++) F.insts.push_back({code, op.targets[j], 0, T, pbits});
            F.cap_sym += (int64_t)k * (c == SP_OP_DEPOLARIZE1 ? 2 : 1);
        } break;
        case SP_OP_DEPOLARIZE2:
            for (uint32_t j = 0; j < k; j += 2) {
                if (op.targets[j] == op.targets[j + 1])
                    return set_error(SP_ERR_INVALID_ARG, "op " + std::to_string(i) + ": DEPOLARIZE2 on one qubit");
                F.insts.push_back({I_DEP2, op.targets[j], op.targets[j + 1], T, pbits});
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

template <typename T>
sp_status dalloc(T **p, size_t count)
{
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_error(SP_ERR_OOM, std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) + " bytes failed");
    }
    return SP_OK;
}

struct Temp {
    std::vector<void *> ptrs;
    ~Temp() { for (void *p : ptrs) cudaFree(p); }
    template <typename T> sp_status alloc(T **p, size_t count)
    {
        sp_status st = dalloc(p, count);
        if (st == SP_OK) ptrs.push_back(*p);
        return st;
    }
};

}  // namespace

#define SP_TRY(x) do { sp_status _s = (x); if (_s != SP_OK) return _s; } while (0)

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

    Temp tmp;
    const int Wq = std::max(1, (n + 31) / 32);
    const int R2 = std::max(32, ((2 * n + 31) / 32) * 32);
    const int64_t cap_sym = F.cap_sym;
    const uint64_t log_cap = 2 * (uint64_t)F.insts.size() + (uint64_t)F.nmeasfam * (2 * (uint64_t)n + 8) +
                             (uint64_t)F.nff * (2 + (uint64_t)n) + 16;

    Inst *d_insts; uint32_t *d_log, *d_inj; uint64_t *d_logpos; uint8_t *d_symrand, *d_recconst;
    TraverseCounts *d_counts; uint32_t *d_gtab = nullptr;
    SP_TRY(tmp.alloc(&d_insts, F.insts.size()));
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
    if (!F.insts.empty())
        SP_CUDA(cudaMemcpyAsync(d_insts, F.insts.data(), F.insts.size() * sizeof(Inst), cudaMemcpyHostToDevice, stream));
    SP_CUDA(cudaMemsetAsync(d_counts, 0, sizeof(TraverseCounts), stream));
    SP_CUDA(cudaMemsetAsync(d_recconst, 0, (size_t)F.nmeas + 1, stream));

    const size_t tab_bytes = 2 * (size_t)Wq * R2 * 4;
    const size_t head_bytes = 64 * 4 + 2048 * 4 + (size_t)R2;
    const bool in_smem = head_bytes + tab_bytes <= 200 * 1024;
    if (!in_smem) SP_TRY(tmp.alloc(&d_gtab, 2 * (size_t)Wq * R2));
    const size_t smem = head_bytes + (in_smem ? tab_bytes : 0);
    SP_CUDA(max_dynamic_smem(k_traverse));
    TravParams tp;
    tp.insts = d_insts; tp.ninst = (int64_t)F.insts.size(); tp.n = n; tp.Wq = Wq; tp.R2 = R2;
    tp.gtab = d_gtab; tp.tab_in_smem = in_smem ? 1 : 0; tp.log = d_log; tp.log_cap = log_cap;
    tp.inj = d_inj; tp.sym_logpos = d_logpos; tp.sym_random = d_symrand;
    tp.chT = P->d_chT; tp.chKind = P->d_chKind; tp.chSym0 = P->d_chSym0; tp.chP = P->d_chP;
    tp.rec_const = d_recconst; tp.counts = d_counts;
    k_traverse<<<1, TRAV_THREADS, smem, stream>>>(tp);
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
        const size_t vsm = (size_t)n * 32 * 4;
        SP_CUDA(max_dynamic_smem(k_replay));
        k_replay<<<(unsigned)nblk, 32, vsm, stream>>>(d_log, hc.log_len, d_inj, Wq, d_logpos,
                                                       hc.nsym, n, P->d_A, P->apitch);
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
        // a detector or observable with a random-measurement symbol is rejected
        uint32_t *d_mask; int *d_bad;
        SP_TRY(tmp.alloc(&d_mask, (size_t)P->apitch));
        SP_TRY(tmp.alloc(&d_bad, 1));
        const int big = 0x7fffffff;
        SP_CUDA(cudaMemcpyAsync(d_bad, &big, 4, cudaMemcpyHostToDevice, stream));
        k_random_mask<<<(unsigned)ceil_div(P->apitch, 128), 128, 0, stream>>>(d_symrand, hc.nsym, d_mask, P->apitch);
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
    // number of random symbols
    {
        std::vector<uint8_t> hk((size_t)P->n_ch);
        if (P->n_ch) SP_CUDA(cudaMemcpy(hk.data(), P->d_chKind, (size_t)P->n_ch, cudaMemcpyDeviceToHost));
        P->n_rand = std::count(hk.begin(), hk.end(), (uint8_t)CK_RANDOM);
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
        SP_TRY(tmp.alloc(&d_fidx, (size_t)tot));
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
    P->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return SP_OK;
}

}  // namespace sp
