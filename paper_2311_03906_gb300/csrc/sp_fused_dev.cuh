// sp_fused_dev.cuh -- device code shared by the fused sampling kernels of
// both fault-draw streams (sp_fused.cu: the per-channel Philox stream;
// sp_grouped.cu: the grouped stream): Philox4x32-10, the channel outcome
// rules, the kernel parameters and one tile of Algorithm 1 "Sampling"
// (Sec. 3.2.3, Eq. sampling) with the draw left to a policy.
#pragma once

#include "sp_internal.h"

namespace sp {

constexpr uint32_t FM = 0xffffffffu;
constexpr uint32_t PH_M0 = 0xD2511F53u, PH_M1 = 0xCD9E8D57u;
constexpr uint32_t PH_W0 = 0x9E3779B9u, PH_W1 = 0xBB67AE85u;
constexpr int FUSED_THREADS = 512;


// Per-shot quantities of the first two Philox rounds that do not depend on
// the channel block.
struct ShotConst {
    uint32_t c1;     // shot hi (counter word 1)
    uint32_t x2;     // round-1 output word 2 = hi(M0*shot_lo) ^ k1
    uint32_t x3;     // round-1 output word 3 = lo(M0*shot_lo)
    uint32_t r2hi;   // hi(M1 * x2), round 2
    uint32_t r2lo;   // lo(M1 * x2), round 2
};

__device__ __forceinline__ ShotConst shot_const(uint64_t shot, uint32_t k1)
{
    ShotConst s;
    const uint64_t p0 = (uint64_t)PH_M0 * (uint32_t)shot;
    s.c1 = (uint32_t)(shot >> 32);
    s.x2 = (uint32_t)(p0 >> 32) ^ k1;
    s.x3 = (uint32_t)p0;
    const uint64_t q = (uint64_t)PH_M1 * s.x2;
    s.r2hi = (uint32_t)(q >> 32);
    s.r2lo = (uint32_t)q;
    return s;
}

// Round keys k + r*W for r = 0..9 (the same for every lane).
struct Keys {
    uint32_t k0[10], k1[10];
};

__device__ __forceinline__ Keys make_keys(uint32_t k0, uint32_t k1)
{
    Keys K;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        K.k0[r] = k0 + (uint32_t)r * PH_W0;
        K.k1[r] = k1 + (uint32_t)r * PH_W1;
    }
    return K;
}

// Rounds 3..10 of Philox4x32-10 from the state (c0, c1, c2, c3) after round 2.
__device__ __forceinline__ void philox_tail(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, const Keys &K,
                                            uint32_t &o0, uint32_t &o1, uint32_t &o2, uint32_t &o3)
{
#pragma unroll
    for (int r = 2; r < 10; r++) {
        const uint64_t p0 = (uint64_t)PH_M0 * c0;
        const uint64_t p1 = (uint64_t)PH_M1 * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ K.k0[r];
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ K.k1[r];
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
    }
    o0 = c0; o1 = c1; o2 = c2; o3 = c3;
}

// Rounds 1..10 of Philox4x32-10 for counter (shot, b): uhi/ulo = M1*b and
// shot_hi = the shot's high word s.c1.  Round 1's output word 0 is
// uhi ^ shot_hi ^ k0 and round 2 multiplies it by M0: that product p is all
// of round 2 that depends on b, so a caller that knows it to be the same in
// several evaluations may compute it once and call philox_from_p.
__device__ __forceinline__ void philox_from_p(const ShotConst &s, uint64_t p, uint32_t ulo, const Keys &K,
                                              uint32_t &o0, uint32_t &o1, uint32_t &o2, uint32_t &o3)
{
    philox_tail(s.r2hi ^ ulo ^ K.k0[1], s.r2lo, (uint32_t)(p >> 32) ^ s.x3 ^ K.k1[1], (uint32_t)p, K, o0, o1, o2, o3);
}

__device__ __forceinline__ void philox_block(const ShotConst &s, uint32_t shot_hi, uint32_t uhi, uint32_t ulo,
                                             const Keys &K, uint32_t &o0, uint32_t &o1, uint32_t &o2, uint32_t &o3)
{
    const uint64_t p = (uint64_t)PH_M0 * (uhi ^ shot_hi ^ K.k0[0]);
    philox_from_p(s, p, ulo, K, o0, o1, o2, o3);
}

// floor(u*m/T) for u < T, exactly: a single-precision estimate (relative
// error below 2^-21, so off by at most one) corrected with integer products.
__device__ __forceinline__ uint32_t cat_index(uint32_t u, uint32_t T, uint32_t m)
{
    const uint64_t um = (uint64_t)u * m;
    uint32_t k = (uint32_t)((float)um * __frcp_rn((float)T));
    k = min(k, m - 1u);
    if ((uint64_t)k * T > um) k--;
    else if ((uint64_t)(k + 1u) * T <= um) k++;
    return k;
}

__device__ __forceinline__ uint32_t chan_bits(uint32_t u, uint32_t T, uint32_t kind)
{
    if (u >= T) return 0u;
    if (kind == CK_DEP1) return cat_index(u, T, 3u) + 1u;
    if (kind == CK_DEP2) return cat_index(u, T, 15u) + 1u;
    return 1u;
}

template <int TW> struct Cols { uint32_t v[TW]; };
template <int TW> struct Shots { ShotConst s[TW]; };

// Fired-event queue of one warp: FUSED_QCAP 32-bit words in shared memory.
// An event is one (channel block, shot) in which some channel may have
// fired: bits 0..4 lane, bit 5 "depolarizing channels only" (its one-symbol
// channels were already applied), then the tile word t (one bit for
// TW <= 2, two for TW = 4), then block - the warp's first block in the
// remaining bits.
// (an enqueue step adds at most 32 events to fewer than 32 and then drains
// 32 whenever 32 are there, so 63 words suffice)
constexpr uint32_t FUSED_QCAP = 64;
constexpr uint32_t EV_DEP_ONLY = 1u << 5;
__host__ __device__ constexpr int event_tbits(int tw) { return tw == 4 ? 2 : 1; }
__host__ __device__ constexpr uint32_t event_max_blocks(int tw) { return 1u << (32 - 6 - event_tbits(tw)); }
// Channel blocks whose compare results are gathered before one vote.
constexpr uint32_t DRAW_GROUP = 8;
static_assert(4 * DRAW_GROUP == 32, "a group's channels map one to one onto the lanes");
// A block is "frequent" when its channels' thresholds add up to at least
// 2^28 (a lane's shot sees one of them fire with probability >= 1/16); its
// blkFilt entry is then FREQUENT, else the largest of its four thresholds.
constexpr uint32_t FREQUENT = 0xFFFFFFFFu;
constexpr uint64_t FREQUENT_SUM = 1ull << 28;

// XOR the word x into tile word t of every measurement row whose own part
// holds symbol s (Eq. sampling restricted to the symbol's column; shared
// atomics, since several symbols of one row may be applied at once).
template <int TW>
__device__ __forceinline__ void xor_column(const uint32_t *__restrict__ colOff, const uint32_t *__restrict__ colRows,
                                           uint32_t s, int t, uint32_t x, uint32_t *Rw)
{
    const uint32_t e = colOff[s + 1];
    for (uint32_t k = colOff[s]; k < e; k++) atomicXor(&Rw[colRows[k] * TW + t], x);
}

// Fired mask of one Philox block: bit i = channel i of the block fired.
__device__ __forceinline__ uint32_t fired4(uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3, const uint4 T)
{
    return (uint32_t)(r0 < T.x) | ((uint32_t)(r1 < T.y) << 1) | ((uint32_t)(r2 < T.z) << 2) |
           ((uint32_t)(r3 < T.w) << 3);
}

struct FusedParams {
    const uint4 *blkT;
    const uint32_t *blkMeta;
    const uint32_t *blkSym0;
    const uint32_t *blkFilt;   // per block: FREQUENT, or the largest of its thresholds
    const uint32_t *colOff;    // [n_sym + 1]: rows of symbol s are colRows[colOff[s] .. colOff[s+1])
    const uint32_t *colRows;   // measurement rows whose own part holds the symbol
    int64_t n_blk, n_rows, n_meas, n_det, n_obs;
    const uint8_t *cflag;      // [n_meas] constant bit of each measurement row's own part
    const uint2 *bItem;        // step B: (row, parent), parents first within a thread
    const uint32_t *bOff;      // [threads + 1]
    const uint32_t *cOff;      // step C: detector/observable t = XOR of measurement rows
    const uint32_t *cRefs;
    uint64_t seed, shot0, nshots;
    Keys keys;                 // Philox round keys of the seed (k_fused reads them from its launch parameters)
    uint64_t *out[3];
    int64_t rows0[3], nrow[3];
    uint32_t aux_off_words;    // the warps' event queues (phase 1), the emit stage (phase 3)
    // grouped draw (stream 2): see sp_grouped.cu
    const uint4 *s2Ch;         // per channel other than random outcomes: {Q, T, first symbol - 1, kind | last << 2}
    const uint4 *s2G;          // per 4 groups of 32 such channels: the groups' thresholds
    const uint32_t *s2Rand;    // per random-outcome channel: its symbol - 1
    uint32_t n_fault, n_grp, n_rnd;
    // phase-2 tables staged in shared memory at this word offset (0 = read
    // from global memory): bItem, bOff, cOff, cRefs, with these counts
    uint32_t tab_off_words, n_items, n_refs;
    uint32_t emit_once;        // 1: phase 3 stages all three record kinds before one copy-out
    // per channel block, for this launch's seed and shot high word (NULL when
    // the launch's shots straddle a multiple of 2^32): {lo(M1 b), lo(p),
    // hi(p), blkFilt[b]} with p = M0 (hi(M1 b) ^ shot hi ^ k0), round 2's
    // product shared by every shot of the launch
    const uint4 *blkConst;
};

// Where phase 2 reads its tables: shared memory when the launch staged them
// (once per persistent CTA), else global memory.
struct FusedTables {
    const uint2 *bItem;
    const uint32_t *bOff, *cOff, *cRefs;
};

__device__ __forceinline__ FusedTables global_tables(const FusedParams &p)
{
    FusedTables t;
    t.bItem = p.bItem; t.bOff = p.bOff; t.cOff = p.cOff; t.cRefs = p.cRefs;
    return t;
}

// Copy the phase-2 tables into shared memory (the whole CTA, then a barrier)
// if the launch asked for it.  Layout from word tab_off_words on: bItem
// (2 words each), bOff (FUSED_THREADS + 1), cOff (targets + 1), cRefs.
__device__ __forceinline__ FusedTables stage_tables(const FusedParams &p, uint32_t *sm)
{
    if (!p.tab_off_words) return global_tables(p);
    uint32_t *base = sm + p.tab_off_words;
    uint2 *bi = reinterpret_cast<uint2 *>(base);
    uint32_t *bo = base + 2 * p.n_items;
    uint32_t *co = bo + FUSED_THREADS + 1;
    const uint32_t ntgt = (uint32_t)(p.n_det + p.n_obs);
    uint32_t *cr = co + ntgt + 1;
    for (uint32_t i = threadIdx.x; i < p.n_items; i += blockDim.x) bi[i] = p.bItem[i];
    for (uint32_t i = threadIdx.x; i <= (uint32_t)FUSED_THREADS; i += blockDim.x) bo[i] = p.bOff[i];
    for (uint32_t i = threadIdx.x; i <= ntgt; i += blockDim.x) co[i] = p.cOff[i];
    for (uint32_t i = threadIdx.x; i < p.n_refs; i += blockDim.x) cr[i] = p.cRefs[i];
    __syncthreads();
    FusedTables t;
    t.bItem = bi; t.bOff = bo; t.cOff = co; t.cRefs = cr;
    return t;
}

// The parameters of one fused launch (host side, sp_fused.cu).
FusedParams fused_params(const sp_program *P, int tw, uint64_t seed, uint64_t shot0, uint64_t nshots,
                         uint64_t *d_meas, uint64_t *d_det, uint64_t *d_obs);

template <int TW> struct TileWord;
template <> struct TileWord<1> {
    typedef uint32_t T;
    __device__ static T zero() { return 0u; }
    __device__ static T ones() { return FM; }
    __device__ static uint32_t get(T v, int) { return v; }
};
template <> struct TileWord<2> {
    typedef uint2 T;
    __device__ static T zero() { return make_uint2(0u, 0u); }
    __device__ static T ones() { return make_uint2(FM, FM); }
    __device__ static uint32_t get(T v, int t) { return t ? v.y : v.x; }
};
template <> struct TileWord<4> {
    typedef uint4 T;
    __device__ static T zero() { return make_uint4(0u, 0u, 0u, 0u); }
    __device__ static T ones() { return make_uint4(FM, FM, FM, FM); }
    __device__ static uint32_t get(T v, int t) { return t == 0 ? v.x : t == 1 ? v.y : t == 2 ? v.z : v.w; }
};
__device__ __forceinline__ uint32_t xorw(uint32_t a, uint32_t b) { return a ^ b; }
__device__ __forceinline__ uint2 xorw(uint2 a, uint2 b) { return make_uint2(a.x ^ b.x, a.y ^ b.y); }
__device__ __forceinline__ uint4 xorw(uint4 a, uint4 b)
{
    return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w);
}

// One tile of 32*TW shots of one program, by the whole CTA of NT threads.
// Ends with a barrier, so the caller may start another tile right away.
// K: the seed's Philox round keys (from the launch parameters, where the
// compiler reads them as constant-bank operands, or computed in registers).
// Draw: the fault draw of phase 1, Draw::run<TW>(p, K, sc, shot_base, warp,
// nwarps, lane, queue, apply), which hands every fired (symbol, tile word,
// shot bits) to apply.
template <int TW, int NT, typename Draw>
__device__ __forceinline__ void fused_tile(const FusedParams &p, const Keys &K, const FusedTables &tab, uint64_t tile,
                                           uint32_t *sm)
{
    typedef TileWord<TW> TWd;
    typedef typename TWd::T W;
    W *Rs = reinterpret_cast<W *>(sm);                       // [n_rows] records, bit-sliced
    uint32_t *aux = sm + p.aux_off_words;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const uint64_t trel = tile * (32u * TW);
    Shots<TW> sc;
#pragma unroll
    for (int t = 0; t < TW; t++) sc.s[t] = shot_const(p.shot0 + trel + 32u * t + lane, Draw::shot_key(p.seed));
    // own parts start from their constants
    for (int64_t j = tid; j < p.n_meas; j += blockDim.x) Rs[j] = p.cflag[j] ? TWd::ones() : TWd::zero();
    __syncthreads();
    // ---- phase 1 + 2A: draw; fired symbols flip the own parts holding them --
    {
        const uint32_t *colOff = p.colOff, *colRows = p.colRows;
        uint32_t *Rw = sm;
        Draw::template run<TW>(p, K, sc, p.shot0 + trel, warp, nwarps, lane, aux + warp * FUSED_QCAP,
                               [=](uint32_t sym, int t, uint32_t word) { xor_column<TW>(colOff, colRows, sym, t, word, Rw); });
    }
    __syncthreads();
    // ---- phase 2B: parent chains, m_j = own part ^ m_parent ---------------
    // (trees are scheduled over FUSED_THREADS lists; a smaller CTA walks
    // several lists, each independent of the others)
    for (int th = tid; th < FUSED_THREADS; th += NT) {
        const uint32_t e = tab.bOff[th + 1];
        for (uint32_t i = tab.bOff[th]; i < e; i++) {
            const uint2 rp = tab.bItem[i];
            Rs[rp.x] = xorw(Rs[rp.x], Rs[rp.y]);
        }
    }
    __syncthreads();
    // ---- phase 2C: detectors and observables from measurement records ------
    for (int64_t t = tid; t < p.n_det + p.n_obs; t += blockDim.x) {
        W acc = TWd::zero();
        for (uint32_t k = tab.cOff[t]; k < tab.cOff[t + 1]; k++) acc = xorw(acc, Rs[tab.cRefs[k]]);
        Rs[p.n_meas + t] = acc;
    }
    __syncthreads();
    // ---- phase 3: emit shot-major records (stage aliases the queues) -------
    // Record kind sg is transposed into the stage, then copied out as
    // contiguous per-shot segments; with emit_once all three kinds share one
    // pass (their stages side by side, one barrier pair), else one pass each.
    uint32_t *stage = aux;
    int soff[3];
    {
        int acc = 0;
#pragma unroll
        for (int sg = 0; sg < 3; sg++) {
            soff[sg] = p.emit_once ? acc : 0;
            acc += 32 * TW * (int)(2 * ((p.nrow[sg] + 63) / 64) + 1);
        }
    }
#pragma unroll
    for (int sg = 0; sg < 3; sg++) {
        {
            uint64_t *dst = p.out[sg];
            const int64_t n = p.nrow[sg];
            if (dst && n) {
                const int64_t row0 = p.rows0[sg];
                const int words32 = (int)(2 * ((n + 63) / 64));
                const int stride = words32 + 1;
                uint32_t *st = stage + soff[sg];
                for (int g = warp; g < words32; g += nwarps) {
                    const int64_t r = 32 * (int64_t)g + lane;
#pragma unroll
                    for (int t = 0; t < TW; t++) {
                        const uint32_t x = r < n ? TWd::get(Rs[row0 + r], t) : 0u;
                        st[(32 * t + lane) * stride + g] = __any_sync(FM, x != 0u) ? transpose32(x, lane) : 0u;
                    }
                }
            }
        }
        if (!p.emit_once || sg == 2) {
            __syncthreads();
#pragma unroll
            for (int sc2 = 0; sc2 < 3; sc2++) {
                if (p.emit_once ? sc2 > sg : sc2 != sg) continue;
                uint64_t *dst = p.out[sc2];
                const int64_t n = p.nrow[sc2];
                if (!dst || n == 0) continue;
                const int words32 = (int)(2 * ((n + 63) / 64));
                const int stride = words32 + 1;
                const uint32_t *st = stage + soff[sc2];
                uint32_t *o32 = reinterpret_cast<uint32_t *>(dst);
                for (int sh = warp; sh < 32 * TW; sh += nwarps) {
                    const uint64_t shot = trel + (uint64_t)sh;
                    if (shot >= p.nshots) continue;
                    uint32_t *o = o32 + shot * (uint64_t)words32;
                    for (int g = lane; g < words32; g += 32) o[g] = st[sh * stride + g];
                }
            }
            __syncthreads();
        }
    }
    // phase 3 may have been skipped (no outputs): keep the tile boundary
    __syncthreads();
}

// Launch shapes: 32- and 64-shot tiles at 512 threads and two CTAs per SM
// (64 registers); U = 2 marks the 64-shot variant compiled for one CTA per
// SM with more registers, U = 3 the 64-shot variant at 256 threads and four
// CTAs per SM.  128-shot tiles (four independent Philox streams
// per thread) run at 256 threads and two CTAs per SM (U = 1) or 512 threads
// and one CTA per SM (U = 2), 128 registers either way.
__host__ __device__ constexpr int fused_threads(int tw, int u) { return (tw == 4 && u == 1) || u == 3 ? 256 : FUSED_THREADS; }
__host__ __device__ constexpr int fused_minb(int tw, int u) { return u == 3 ? 4 : (u == 2 && tw != 1 ? 1 : 2); }

}  // namespace sp
