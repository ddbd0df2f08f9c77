// sp_fused.cu -- the sampling hot path fused into one persistent kernel.
//
// Algorithm 1 "Sampling" (arXiv 2311.03906, Sec. 3.2.3, Eq. sampling) for a
// tile of 32*TW shots per CTA iteration, entirely in shared memory:
//   phase 1  draw: Philox4x32-10 keyed by (seed, shot, channel/4); each warp
//            owns a contiguous range of 4-channel blocks, lane = shot.  Per
//            block it draws and compares with the four thresholds; per group
//            of 8 blocks the fired bits of a lane's shots are gathered into
//            one word per tile word.  Faults are rare at circuit-level noise:
//            each (block, shot) in which some channel fired is queued as one
//            event, and the queue is drained by all lanes of the warp
//            together (a depolarizing channel draws its category again);
//            each fired symbol XORs its shot bit into the rows holding it;
//   phase 2  product: (A) every measurement row's own part, c'_j ^ XOR of
//            its delta symbols, applied symbol by symbol in phase 1; (B) the
//            parent chains m_j ^= m_parent; (C) detectors and observables as
//            XORs of their measurement records, which is their definition;
//   phase 3  emit: 32x32 warp transposes turn the bit-sliced rows into
//            shot-major packed words, staged in shared memory and written as
//            contiguous per-shot segments.
// Nothing but the records touches HBM.  The staged path (fault bits to global
// memory) draws with a dense variant that transposes 32-symbol groups.
//
// Philox per (shot, channel block b): counter (shot lo, shot hi, b, 0).
// Round 1's product M1*b is the same for every lane (one per warp), and the
// products M0*(shot lo) of round 1 and M1*(hi0 ^ k1) of round 2 do not depend
// on b, so they are computed once per shot; round 2's M0 product depends on b
// and the shot's high word only, so a tile whose shots share that word
// computes it once per block: 16 of the 20 wide multiplies of a block remain
// per (shot, block).
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <tuple>
#include <vector>

#include "sp_fused_dev.cuh"

namespace sp {

// Draw the symbols of blocks [b0, b1) for TW shots per lane (shot words
// w_t = 32-shot groups).  Each flushed 32-symbol column group is handed to
// sink(symbol base, lane's column words[TW]) with the lane's symbol = base+lane.

template <int TW, int U, typename Sink>
__device__ __forceinline__ void draw_blocks(const uint4 *__restrict__ blkT, const uint32_t *__restrict__ blkMeta,
                                            uint32_t b0, uint32_t b1, uint32_t sym_begin, const Shots<TW> sc,
                                            uint32_t k0, uint32_t k1, int lane, Sink sink)
{
    const Keys K = make_keys(k0, k1);
    uint64_t acc[TW];
#pragma unroll
    for (int t = 0; t < TW; t++) acc[t] = 0;
    uint32_t fill = 0, base = sym_begin;
    auto flush = [&]() {
        Cols<TW> col;
#pragma unroll
        for (int t = 0; t < TW; t++) {
            const uint32_t lo = (uint32_t)acc[t];
            col.v[t] = __any_sync(FM, lo != 0u) ? transpose32(lo, lane) : 0u;
            acc[t] >>= 32;
        }
        sink(base, col);
        fill -= 32;
        base += 32;
    };
    // U blocks per iteration: U*TW independent Philox evaluations per lane.
    // fill stays below 32 between iterations and a block adds at most 16
    // symbols, so U <= 2 keeps every inserted bit inside the 64-bit word.
    static_assert(U == 1 || U == 2, "at most two blocks per iteration");
    uint32_t b = b0;
    // round-1 product M1*b, advanced by addition (it is the same in all lanes)
    uint64_t ub = (uint64_t)PH_M1 * b;
    for (; b + U <= b1; b += U) {
        uint4 T[U];
        uint32_t meta[U];
        uint32_t r[U][TW][4];
        bool fire = false;
#pragma unroll
        for (int v = 0; v < U; v++) {
            T[v] = blkT[b + v];
            meta[v] = blkMeta[b + v];
            const uint64_t uv = ub + (uint64_t)v * PH_M1;
#pragma unroll
            for (int t = 0; t < TW; t++) {
                philox_block(sc.s[t], sc.s[t].c1, (uint32_t)(uv >> 32), (uint32_t)uv, K, r[v][t][0], r[v][t][1], r[v][t][2], r[v][t][3]);
                fire |= (r[v][t][0] < T[v].x) | (r[v][t][1] < T[v].y) | (r[v][t][2] < T[v].z) | (r[v][t][3] < T[v].w);
            }
        }
        ub += (uint64_t)U * PH_M1;
        // Faults are rare: one vote decides whether any lane needs the
        // channel bits of these blocks; then only the channels that fired in
        // some lane are visited.
        if (__any_sync(FM, fire)) {
            uint32_t at = fill;
#pragma unroll
            for (int v = 0; v < U; v++) {
                uint32_t fm[TW];
                uint32_t any = 0;
#pragma unroll
                for (int t = 0; t < TW; t++) {
                    fm[t] = (uint32_t)(r[v][t][0] < T[v].x) | ((uint32_t)(r[v][t][1] < T[v].y) << 1) |
                            ((uint32_t)(r[v][t][2] < T[v].z) << 2) | ((uint32_t)(r[v][t][3] < T[v].w) << 3);
                    any |= fm[t];
                }
                uint32_t wm = __reduce_or_sync(FM, any);
                while (wm) {
                    const int i = __ffs(wm) - 1;
                    wm &= wm - 1;
                    const uint32_t kind = (meta[v] >> (2 * i)) & 3u;
                    const uint32_t off = at + ((meta[v] >> (8 + 4 * i)) & 15u);
                    const uint32_t Ti = i == 0 ? T[v].x : i == 1 ? T[v].y : i == 2 ? T[v].z : T[v].w;
#pragma unroll
                    for (int t = 0; t < TW; t++) {
                        if ((fm[t] >> i) & 1u) {
                            const uint32_t u = i == 0 ? r[v][t][0] : i == 1 ? r[v][t][1] : i == 2 ? r[v][t][2] : r[v][t][3];
                            acc[t] |= (uint64_t)chan_bits(u, Ti, kind) << off;
                        }
                    }
                }
                at += meta[v] >> 24;
            }
        }
#pragma unroll
        for (int v = 0; v < U; v++) fill += meta[v] >> 24;
        if (fill >= 32) flush();
    }
    for (; b < b1; b++) {
        const uint4 T = blkT[b];
        const uint32_t meta = blkMeta[b];
        const uint64_t ub = (uint64_t)PH_M1 * b;
        const uint32_t Ts[4] = {T.x, T.y, T.z, T.w};
#pragma unroll
        for (int t = 0; t < TW; t++) {
            uint32_t r[4];
            philox_block(sc.s[t], sc.s[t].c1, (uint32_t)(ub >> 32), (uint32_t)ub, K, r[0], r[1], r[2], r[3]);
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const uint32_t kind = (meta >> (2 * i)) & 3u;
                const uint32_t off = fill + ((meta >> (8 + 4 * i)) & 15u);
                acc[t] |= (uint64_t)chan_bits(r[i], Ts[i], kind) << off;
            }
        }
        fill += meta >> 24;
        if (fill >= 32) flush();
    }
    if (fill > 0) {
        Cols<TW> col;
#pragma unroll
        for (int t = 0; t < TW; t++) {
            const uint32_t lo = (uint32_t)acc[t];
            col.v[t] = __any_sync(FM, lo != 0u) ? transpose32(lo, lane) : 0u;
        }
        sink(base, col);
    }
}

// Apply the queued events e = lane, lane+32, ... < n: recompute the event's
// Philox block, compare its four words with the thresholds, turn each fired
// channel into its symbol bits and hand each (symbol, tile word, shot bit)
// to apply.
template <int TW, typename Apply>
__device__ __forceinline__ void drain_fired(const uint32_t *q, uint32_t n, const uint4 *__restrict__ blkT,
                                            const uint32_t *__restrict__ blkMeta, const uint32_t *__restrict__ blkSym0,
                                            uint32_t b0, uint64_t shot_base, const Keys &K, uint32_t k1, int lane,
                                            const Apply &apply)
{
    __syncwarp();
    constexpr int TB = event_tbits(TW);
    for (uint32_t e = lane; e < n; e += 32) {
        const uint32_t ev = q[e];
        const uint32_t b = b0 + (ev >> (6 + TB));
        const int t = (ev >> 6) & ((1u << TB) - 1u);
        const uint32_t ln = ev & 31u;
        const ShotConst s = shot_const(shot_base + 32u * (uint32_t)t + ln, k1);
        const uint64_t ub = (uint64_t)PH_M1 * b;
        uint32_t r0, r1, r2, r3;
        philox_block(s, s.c1, (uint32_t)(ub >> 32), (uint32_t)ub, K, r0, r1, r2, r3);
        const uint4 T = blkT[b];
        const uint32_t meta = blkMeta[b], s0 = blkSym0[b];
        uint32_t fmask = fired4(r0, r1, r2, r3, T);
        if (ev & EV_DEP_ONLY) {
            const uint32_t dep = (((meta >> 0) & 3u) ? 1u : 0u) | (((meta >> 2) & 3u) ? 2u : 0u) |
                                 (((meta >> 4) & 3u) ? 4u : 0u) | (((meta >> 6) & 3u) ? 8u : 0u);
            fmask &= dep;
        }
        while (fmask) {
            const int i = __ffs(fmask) - 1;
            fmask &= fmask - 1;
            const uint32_t kind = (meta >> (2 * i)) & 3u;
            const uint32_t off = s0 + ((meta >> (8 + 4 * i)) & 15u);
            const uint32_t Ti = i == 0 ? T.x : i == 1 ? T.y : i == 2 ? T.z : T.w;
            const uint32_t u = i == 0 ? r0 : i == 1 ? r1 : i == 2 ? r2 : r3;
            uint32_t val = chan_bits(u, Ti, kind);
            while (val) {
                const int j = __ffs(val) - 1;
                val &= val - 1;
                apply(off + (uint32_t)j, t, 1u << ln);
            }
        }
    }
    __syncwarp();
}

// Phase 1 with the product folded in, for blocks [b0, b1) and 32*TW shots:
// every fired symbol XORs its bit-sliced word (bit = shot in the tile) into
// the rows Rw (TW 32-bit words per row) whose own part holds it.  Blocks go
// in groups of DRAW_GROUP (32 channels), with one of two treatments chosen
// per group by a warp vote on the blocks' blkFilt entries:
//  - rare groups (every block's thresholds add up to less than 2^28; at
//    circuit-level noise all of them): per block and shot only the least of
//    the four Philox words is compared, with the block's largest threshold,
//    which no fired channel can miss; each (block, shot) that passes is
//    queued as an event, and the drain recomputes its Philox block and
//    compares channel by channel, so the records are exact;
//  - frequent groups (some block holds a channel that fires often, such as a
//    random outcome at T = 2^31): every channel is compared; a one-symbol
//    channel's fired shots come out of a 32x32 transpose (lane j = channel j
//    of the group) as one column word per tile word, and a depolarizing
//    channel is queued as an event that applies only its depolarizing
//    channels.
// The queue is drained by all 32 lanes together when it fills and at the end.
// UHI: every shot of the tile has the same high counter word c1u, so round
// 2's M0 product is the same in all lanes and tile words.
// BC: the launch supplies blkConst (every shot shares the high word c1u).
template <int TW, bool UHI, bool BC, typename Apply>
__device__ __forceinline__ void draw_group_impl(const uint4 *__restrict__ blkT, const uint32_t *__restrict__ blkMeta,
                                                const uint32_t *__restrict__ blkSym0,
                                                const uint32_t *__restrict__ blkFilt,
                                                const uint4 *__restrict__ blkConst, uint32_t b0, uint32_t b1,
                                                const Shots<TW> sc, uint64_t shot_base, const Keys &K, uint32_t k1,
                                                int lane, uint32_t *q, const Apply &apply)
{
    static_assert(TW == 1 || TW == 2 || TW == 4, "one, two or four tile words");
    constexpr int TB = event_tbits(TW);
    const uint32_t c1u = (uint32_t)(shot_base >> 32);
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t cnt = 0;
    // queue the events flagged in m (bit k = block g + k), one per set bit;
    // as soon as 32 are queued they are applied by one lane each, so that
    // the drains' memory latency overlaps the other warps' draws
    auto enqueue = [&](uint32_t g, int t, uint32_t m, uint32_t flags, int stride) {
        while (__any_sync(FM, m != 0u)) {
            const uint32_t k = m ? (uint32_t)(__ffs(m) - 1) / (uint32_t)stride : 0u;
            const uint32_t bal = __ballot_sync(FM, m != 0u);
            if (m)
                q[cnt + __popc(bal & lt)] = ((g + k - b0) << (6 + TB)) | ((uint32_t)t << 6) | flags | (uint32_t)lane;
            cnt += __popc(bal);
            m &= ~(((1u << stride) - 1u) << (stride * k));
            if (cnt >= 32u) {
                drain_fired<TW>(q, 32u, blkT, blkMeta, blkSym0, b0, shot_base, K, k1, lane, apply);
                cnt -= 32u;
                // the rest (fewer than 32) moves to the front
                const uint32_t rest = (uint32_t)lane < cnt ? q[32 + lane] : 0u;
                __syncwarp();
                if ((uint32_t)lane < cnt) q[lane] = rest;
                __syncwarp();
            }
        }
    };
    // rare block g+kk from its launch constants: one uniform load
    auto step_rare_bc = [&](uint32_t g, uint32_t kk, uint32_t (&word)[TW]) {
        const uint4 bc = blkConst[g + kk];
        const uint64_t p = ((uint64_t)bc.z << 32) | bc.y;
#pragma unroll
        for (int t = 0; t < TW; t++) {
            uint32_t r0, r1, r2, r3;
            philox_from_p(sc.s[t], p, bc.x, K, r0, r1, r2, r3);
            if (min(min(r0, r1), min(r2, r3)) < bc.w) word[t] |= 1u << kk;
        }
    };
    // rare block g+kk: bit kk of word[t] = the least of the shot's four
    // words is below tm, the block's largest threshold
    auto step_rare = [&](uint32_t kk, uint64_t ub, uint32_t tm, uint32_t (&word)[TW]) {
        const uint32_t uhi = (uint32_t)(ub >> 32), ulo = (uint32_t)ub;
        uint64_t p = 0;
        if (UHI) p = (uint64_t)PH_M0 * (uhi ^ c1u ^ K.k0[0]);
#pragma unroll
        for (int t = 0; t < TW; t++) {
            if (!UHI) p = (uint64_t)PH_M0 * (uhi ^ sc.s[t].c1 ^ K.k0[0]);
            uint32_t r0, r1, r2, r3;
            philox_from_p(sc.s[t], p, ulo, K, r0, r1, r2, r3);
            if (min(min(r0, r1), min(r2, r3)) < tm) word[t] |= 1u << kk;
        }
    };
    // frequent block g+kk: bit 4*kk+i of word[t] = channel i fired in shot t
    auto step_exact = [&](uint32_t g, uint32_t kk, uint64_t ub, uint32_t (&word)[TW]) {
        const uint4 T = blkT[g + kk];
        const uint32_t uhi = (uint32_t)(ub >> 32), ulo = (uint32_t)ub;
        const uint32_t bit = 1u << (4 * kk);
        uint64_t p = 0;
        if (UHI) p = (uint64_t)PH_M0 * (uhi ^ c1u ^ K.k0[0]);
#pragma unroll
        for (int t = 0; t < TW; t++) {
            if (!UHI) p = (uint64_t)PH_M0 * (uhi ^ sc.s[t].c1 ^ K.k0[0]);
            uint32_t r0, r1, r2, r3;
            philox_from_p(sc.s[t], p, ulo, K, r0, r1, r2, r3);
            if (r0 < T.x) word[t] |= bit;
            if (r1 < T.y) word[t] |= bit << 1;
            if (r2 < T.z) word[t] |= bit << 2;
            if (r3 < T.w) word[t] |= bit << 3;
        }
    };
    constexpr uint32_t ALL = (1u << DRAW_GROUP) - 1u;
    for (uint32_t g = b0; g < b1; g += DRAW_GROUP) {
        const uint32_t nb = min(DRAW_GROUP, b1 - g);
        // lane k < nb holds block g+k's filter threshold
        const uint32_t filt = (uint32_t)lane < nb ? blkFilt[g + lane] : 0u;
        // blocks with a channel that can fire (a zero filter entry: every
        // threshold is zero, so no channel of the block fires in any shot and
        // its Philox words are not needed)
        const uint32_t act = __ballot_sync(FM, filt != 0u);
        if (!act) continue;
        const uint64_t ug = (uint64_t)PH_M1 * g;
        uint32_t word[TW];
#pragma unroll
        for (int t = 0; t < TW; t++) word[t] = 0u;
        if (!__any_sync(FM, filt == FREQUENT)) {
            if (BC && act == ALL) {
#pragma unroll
                for (uint32_t kk = 0; kk < DRAW_GROUP; kk++) step_rare_bc(g, kk, word);
            } else if (act == ALL) {
#pragma unroll
                for (uint32_t kk = 0; kk < DRAW_GROUP; kk++)
                    step_rare(kk, ug + (uint64_t)kk * PH_M1, __shfl_sync(FM, filt, kk), word);
            } else {
#pragma unroll 1
                for (uint32_t m = act; m; m &= m - 1u) {
                    const uint32_t kk = (uint32_t)__ffs(m) - 1u;
                    if (BC) step_rare_bc(g, kk, word);
                    else step_rare(kk, ug + (uint64_t)kk * PH_M1, __shfl_sync(FM, filt, kk), word);
                }
            }
#pragma unroll
            for (int t = 0; t < TW; t++) enqueue(g, t, word[t], 0u, 1);
            continue;
        }
        // ---- frequent group: lane j stands for channel j&3 of block g + j/4
        uint32_t jmeta = 0, js0 = 0;
        if ((uint32_t)(lane >> 2) < nb) {
            jmeta = blkMeta[g + (lane >> 2)];
            js0 = blkSym0[g + (lane >> 2)];
        }
        if (act == ALL) {
#pragma unroll
            for (uint32_t kk = 0; kk < DRAW_GROUP; kk++) step_exact(g, kk, ug + (uint64_t)kk * PH_M1, word);
        } else {
#pragma unroll 1
            for (uint32_t m = act; m; m &= m - 1u) {
                const uint32_t kk = (uint32_t)__ffs(m) - 1u;
                step_exact(g, kk, ug + (uint64_t)kk * PH_M1, word);
            }
        }
        uint32_t any = 0;
#pragma unroll
        for (int t = 0; t < TW; t++) any |= word[t];
        const uint32_t wm = __reduce_or_sync(FM, any);
        if (!wm) continue;
        const int i = lane & 3;
        const uint32_t kind = (jmeta >> (2 * i)) & 3u;
        const bool mine = (wm >> lane) & 1u;
        const bool is_dep = kind == CK_DEP1 || kind == CK_DEP2;
        const uint32_t dep = __ballot_sync(FM, mine && is_dep);
        if (wm & ~dep) {
            const uint32_t sym = js0 + ((jmeta >> (8 + 4 * i)) & 15u);
#pragma unroll
            for (int t = 0; t < TW; t++) {
                const uint32_t col = transpose32(word[t], lane);
                if (mine && !is_dep && col) apply(sym, t, col);
            }
        }
        if (dep) {
#pragma unroll
            for (int t = 0; t < TW; t++) enqueue(g, t, word[t] & dep, EV_DEP_ONLY, 4);
        }
    }
    drain_fired<TW>(q, cnt, blkT, blkMeta, blkSym0, b0, shot_base, K, k1, lane, apply);
}

template <int TW, typename Apply>
__device__ __forceinline__ void draw_scatter(const uint4 *__restrict__ blkT, const uint32_t *__restrict__ blkMeta,
                                             const uint32_t *__restrict__ blkSym0, const uint32_t *__restrict__ blkFilt,
                                             const uint4 *__restrict__ blkConst, uint32_t b0, uint32_t b1,
                                             const Shots<TW> sc, uint64_t shot_base, const Keys &K, uint32_t k1,
                                             int lane, uint32_t *q, const Apply &apply)
{
    // a tile straddles a multiple of 2^32 shots only if shot0 is unaligned;
    // blkConst is given only when no tile of the launch does
    if (blkConst)
        draw_group_impl<TW, true, true>(blkT, blkMeta, blkSym0, blkFilt, blkConst, b0, b1, sc, shot_base, K, k1, lane,
                                        q, apply);
    else if ((shot_base >> 32) == ((shot_base + 32u * TW - 1u) >> 32))
        draw_group_impl<TW, true, false>(blkT, blkMeta, blkSym0, blkFilt, blkConst, b0, b1, sc, shot_base, K, k1,
                                         lane, q, apply);
    else
        draw_group_impl<TW, false, false>(blkT, blkMeta, blkSym0, blkFilt, blkConst, b0, b1, sc, shot_base, K, k1,
                                          lane, q, apply);
}

// The launch constants of every channel block of every batch member (shots
// from 0, so the high word is 0): thread i is block i - blkStart[m] of member
// m, found by binary search over the members' cumulative block counts.
__global__ void __launch_bounds__(256) k_block_consts_batch(const FusedParams *__restrict__ params, int nprog,
                                                            const uint64_t *__restrict__ blkEnd)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= blkEnd[nprog - 1]) return;
    int lo = 0, hi = nprog - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (blkEnd[mid] > i) hi = mid; else lo = mid + 1;
    }
    const FusedParams &p = params[lo];
    if (!p.blkConst) return;   // this member draws without launch constants
    const uint32_t b = (uint32_t)(i - (lo ? blkEnd[lo - 1] : 0ull));
    const uint64_t ub = (uint64_t)PH_M1 * b;
    const uint64_t pp = (uint64_t)PH_M0 * ((uint32_t)(ub >> 32) ^ (uint32_t)p.seed);
    const_cast<uint4 *>(p.blkConst)[b] = make_uint4((uint32_t)ub, (uint32_t)pp, (uint32_t)(pp >> 32), p.blkFilt[b]);
}

// The launch constants of every channel block (see FusedParams::blkConst).
__global__ void __launch_bounds__(256) k_block_consts(int64_t n_blk, uint32_t k0, uint32_t c1u,
                                                      const uint32_t *__restrict__ blkFilt, uint4 *__restrict__ out)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_blk) return;
    const uint64_t ub = (uint64_t)PH_M1 * (uint32_t)b;
    const uint64_t p = (uint64_t)PH_M0 * ((uint32_t)(ub >> 32) ^ c1u ^ k0);
    out[b] = make_uint4((uint32_t)ub, (uint32_t)p, (uint32_t)(p >> 32), blkFilt[b]);
}

// The per-channel Philox stream (the default draw): warp w of the CTA owns
// the channel blocks [b0, b1) of an even split.
struct DrawPerChannel {
    __device__ static uint32_t shot_key(uint64_t seed) { return (uint32_t)(seed >> 32); }
    template <int TW, typename Apply>
    __device__ static void run(const FusedParams &p, const Keys &K, const Shots<TW> &sc, uint64_t shot_base, int warp,
                               int nwarps, int lane, uint32_t *q, const Apply &apply)
    {
        const uint32_t b0 = (uint32_t)((uint64_t)warp * (uint64_t)p.n_blk / (uint64_t)nwarps);
        const uint32_t b1 = (uint32_t)((uint64_t)(warp + 1) * (uint64_t)p.n_blk / (uint64_t)nwarps);
        draw_scatter<TW>(p.blkT, p.blkMeta, p.blkSym0, p.blkFilt, p.blkConst, b0, b1, sc, shot_base, K,
                         (uint32_t)(p.seed >> 32), lane, q, apply);
    }
};

template <int TW, int U>
__global__ void __launch_bounds__(fused_threads(TW, U), fused_minb(TW, U)) k_fused(FusedParams p)
{
    extern __shared__ __align__(16) uint32_t sm[];
    const uint64_t per_tile = 32u * TW;
    const uint64_t ntiles = (p.nshots + per_tile - 1) / per_tile;
    const FusedTables tab = stage_tables(p, sm);
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
        fused_tile<TW, fused_threads(TW, U), DrawPerChannel>(p, p.keys, tab, tile, sm);
}

// Batched form: many programs in one persistent launch per launch shape.
// Work items are (program, tile) pairs handed out in order by an atomic
// counter; items of member i are [tileEnd[i-1], tileEnd[i]).  Every member
// of one launch uses the tile size and launch shape its own build-time
// autotuner chose (TW, U); the launcher orders the members by decreasing
// cost per tile so the tail is made of the cheapest items.
template <int TW, int U>
__global__ void __launch_bounds__(fused_threads(TW, U), fused_minb(TW, U))
    k_fused_batch(const FusedParams *__restrict__ progs, int nprog, const uint64_t *__restrict__ tileEnd,
                  unsigned long long *counter)
{
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ unsigned long long s_item;
    const uint64_t total = tileEnd[nprog - 1];
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1ull);
        __syncthreads();
        const uint64_t item = s_item;
        __syncthreads();
        if (item >= total) break;
        int lo = 0, hi = nprog - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (tileEnd[mid] > item) hi = mid; else lo = mid + 1;
        }
        // parameters in global memory: the round keys are computed into registers
        const uint64_t seed = progs[lo].seed;
        const Keys K = make_keys((uint32_t)seed, (uint32_t)(seed >> 32));
        fused_tile<TW, fused_threads(TW, U), DrawPerChannel>(progs[lo], K, global_tables(progs[lo]),
                                                             item - (lo ? tileEnd[lo - 1] : 0ull), sm);
    }
}

// Staged draw: fault bits to global memory, bit-sliced [symbol][32-shot word].
// Block = 8 warps; warp = one 32-shot word over all channel blocks.
// Block = 8 warps; warp = one 32-shot word over the channel blocks of range
// blockIdx.y (gridDim.y even ranges, so that few shots still fill the GPU).
// A range writes only its own symbols' rows of B: its last, partial set of
// 32 stops at the next range's first symbol.
__global__ void __launch_bounds__(256) k_draw_staged(const uint4 *__restrict__ blkT,
                                                     const uint32_t *__restrict__ blkMeta,
                                                     const uint32_t *__restrict__ blkSym0, int64_t n_blk,
                                                     int64_t n_sym, uint64_t seed, uint64_t shot0, int64_t nwords,
                                                     uint32_t *__restrict__ B, int64_t bpitch)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (w >= nwords) return;
    const uint32_t b0 = (uint32_t)((uint64_t)n_blk * blockIdx.y / gridDim.y);
    const uint32_t b1 = (uint32_t)((uint64_t)n_blk * (blockIdx.y + 1) / gridDim.y);
    if (b0 >= b1) return;
    const uint32_t s_begin = blkSym0[b0];
    const int64_t s_end = b1 < (uint64_t)n_blk ? (int64_t)blkSym0[b1] : n_sym;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    Shots<1> sc;
    sc.s[0] = shot_const(shot0 + (uint64_t)w * 32u + (uint64_t)lane, k1);
    draw_blocks<1, 2>(blkT, blkMeta, b0, b1, s_begin, sc, k0, k1, lane,
                   [=](uint32_t base, const Cols<1> col) {
                       if ((int64_t)base + lane < s_end) B[(size_t)(base + lane) * bpitch + w] = col.v[0];
                   });
}

// The draw fused with the sparse product in global memory, for records
// that fit in L2: warp = 64 shots (two 32-shot words) over one range of
// channel blocks (blockIdx.y), with the fused kernel's draw (least-word
// filter, events resolved 32 at a time); every fired symbol's shot word is
// XORed straight into the records of the rows holding it (the full rows by
// symbol; rec pre-filled with the rows' constants, word-major: word w of row
// j at rec[w * nrows + j]), by atomics in L2.
__global__ void __launch_bounds__(256, 4) k_draw_push(const uint4 *__restrict__ blkT,
                                                      const uint32_t *__restrict__ blkMeta,
                                                      const uint32_t *__restrict__ blkSym0,
                                                      const uint32_t *__restrict__ blkFilt,
                                                      const uint4 *__restrict__ blkConst, int64_t n_blk,
                                                      uint64_t seed, const Keys K, uint64_t shot0, int64_t nwords,
                                                      const uint32_t *__restrict__ colOff,
                                                      const uint32_t *__restrict__ colRows, uint32_t *rec,
                                                      int64_t nrows)
{
    __shared__ uint32_t q[8 * FUSED_QCAP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * 8 + warp;      // words 2gw and 2gw+1
    if (2 * gw >= nwords) return;
    const uint32_t k1 = (uint32_t)(seed >> 32);
    const uint64_t shot_base = shot0 + 64u * (uint64_t)gw;
    Shots<2> sc;
#pragma unroll
    for (int t = 0; t < 2; t++) sc.s[t] = shot_const(shot_base + 32u * t + lane, k1);
    const bool has2 = 2 * gw + 1 < nwords;
    const uint64_t ngrp = ((uint64_t)n_blk + DRAW_GROUP - 1) / DRAW_GROUP;
    const uint32_t b0 = (uint32_t)(ngrp * blockIdx.y / gridDim.y) * DRAW_GROUP;
    const uint64_t e1 = ngrp * (blockIdx.y + 1) / gridDim.y * DRAW_GROUP;
    const uint32_t b1 = (uint32_t)(e1 < (uint64_t)n_blk ? e1 : (uint64_t)n_blk);
    if (b0 >= b1) return;
    // word 2gw of row j at rec[2gw * nrows + j], word 2gw+1 nrows later (the
    // launcher keeps nwords * nrows below 2^32)
    const uint32_t nr = (uint32_t)nrows, w0 = (uint32_t)(2 * gw) * nr;
    draw_scatter<2>(blkT, blkMeta, blkSym0, blkFilt, blkConst, b0, b1, sc, shot_base, K, k1, lane,
                    q + warp * FUSED_QCAP,
                    [=](uint32_t sym, int t, uint32_t word) {
                        if (t == 1 && !has2) return;
                        const uint32_t base = w0 + (t ? nr : 0u);
                        const uint32_t e = colOff[sym + 1];
                        for (uint32_t k = colOff[sym]; k < e; k++) atomicXor(&rec[base + colRows[k]], word);
                    });
}

sp_status launch_draw_push(const sp_program *P, uint64_t seed, uint64_t shot0, int64_t nwords, uint32_t *rec,
                           cudaStream_t s)
{
    if (P->n_blk == 0 || nwords == 0) return SP_OK;
    // a warp's queued events address the blocks of its range (at most all)
    if ((uint64_t)P->n_blk >= event_max_blocks(2))
        return set_error(SP_ERR_INVALID_ARG, "too many channel blocks for the staged draw");
    if ((uint64_t)nwords * (uint64_t)P->n_rows >= (1ull << 32))
        return set_error(SP_ERR_INVALID_ARG, "records too large for the push draw");
    // about four waves of warps (4 CTAs of 8 warps per SM), each range keeping at least 64 groups
    const int64_t ctas = ceil_div(ceil_div(nwords, 2), 8);
    const int64_t want = 4 * 4 * (int64_t)std::max(P->num_sms, 1);
    const int64_t ngrp = ceil_div(P->n_blk, (int64_t)DRAW_GROUP);
    const int64_t ranges = std::max<int64_t>(1, std::min<int64_t>({ceil_div(want, ctas), ngrp / 64, 65535}));
    // the round keys as launch parameters (constant-bank operands), and the
    // launch's block constants when all its shots share a high word
    Keys K;
    for (int r = 0; r < 10; r++) {
        K.k0[r] = (uint32_t)seed + (uint32_t)r * PH_W0;
        K.k1[r] = (uint32_t)(seed >> 32) + (uint32_t)r * PH_W1;
    }
    const uint4 *consts = nullptr;
    if (P->d_blkConst && (shot0 >> 32) == ((shot0 + 32u * (uint64_t)nwords - 1u) >> 32)) {
        k_block_consts<<<(unsigned)ceil_div(P->n_blk, 256), 256, 0, s>>>(P->n_blk, (uint32_t)seed,
                                                                        (uint32_t)(shot0 >> 32), P->d_blkFilt,
                                                                        P->d_blkConst);
        SP_CUDA(cudaGetLastError());
        consts = P->d_blkConst;
    }
    k_draw_push<<<dim3((unsigned)ctas, (unsigned)ranges), 256, 0, s>>>(
        P->d_blkT, P->d_blkMeta, P->d_blkSym0, P->d_blkFilt, consts, P->n_blk, seed, K, shot0, nwords,
        P->d_colFullOff, P->d_colFullRows, rec, P->n_rows);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

// Shot-major draw for the dense products.  Word w of shot 32g+l (entries
// 32w..32w+31 of (s_0, s_1, ...), b_0 = 1 of Eq. sampling) is stored at
// Bd[(g * bpitch + w) * 32 + l].  k_dense_fill writes the constant bit and
// zeroes the rest; k_draw_dense runs the grouped draw for 64 shots per warp
// over one range of channel blocks (blockIdx.y of gridDim.y even ranges, so
// that small shot counts still fill the GPU) and sets the bit of each fired
// symbol in the shots that drew it (global atomics: faults are rare, and
// warps of other ranges may share a word).
__global__ void __launch_bounds__(256) k_dense_fill(uint32_t *__restrict__ Bd, int64_t bpitch, int64_t nvec)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nvec) return;
    const int64_t w = (i / 8) % bpitch;   // 8 uint4 per 32-lane word
    const uint32_t v = w == 0 ? 1u : 0u;
    reinterpret_cast<uint4 *>(Bd)[i] = make_uint4(v, v, v, v);
}

__global__ void __launch_bounds__(256, 4) k_draw_dense(const uint4 *__restrict__ blkT,
                                                       const uint32_t *__restrict__ blkMeta,
                                                       const uint32_t *__restrict__ blkSym0,
                                                       const uint32_t *__restrict__ blkFilt,
                                                       const uint4 *__restrict__ blkConst, int64_t n_blk,
                                                       uint64_t seed, const Keys K, uint64_t shot0, int64_t ngroups,
                                                       uint32_t *__restrict__ Bd, int64_t bpitch)
{
    __shared__ uint32_t q[8 * FUSED_QCAP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * 8 + warp;      // groups 2gw and 2gw+1
    if (2 * gw >= ngroups) return;
    const uint32_t k1 = (uint32_t)(seed >> 32);
    const uint64_t shot_base = shot0 + 64u * (uint64_t)gw;
    Shots<2> sc;
#pragma unroll
    for (int t = 0; t < 2; t++) sc.s[t] = shot_const(shot_base + 32u * t + lane, k1);
    uint32_t *base = Bd + (size_t)(2 * gw) * (size_t)bpitch * 32u;
    const bool has2 = 2 * gw + 1 < ngroups;
    // this CTA's range of channel blocks, in whole groups of DRAW_GROUP
    const uint64_t ngrp = ((uint64_t)n_blk + DRAW_GROUP - 1) / DRAW_GROUP;
    const uint32_t b0 = (uint32_t)(ngrp * blockIdx.y / gridDim.y) * DRAW_GROUP;
    const uint64_t e1 = ngrp * (blockIdx.y + 1) / gridDim.y * DRAW_GROUP;
    const uint32_t b1 = (uint32_t)(e1 < (uint64_t)n_blk ? e1 : (uint64_t)n_blk);
    if (b0 >= b1) return;
    // offsets within this warp's two shot groups (2 * bpitch * 32 words,
    // below 2^32: the launcher checks)
    const uint32_t gstride = (uint32_t)bpitch * 32u;
    draw_scatter<2>(blkT, blkMeta, blkSym0, blkFilt, blkConst, b0, b1, sc, shot_base, K, k1, lane,
                    q + warp * FUSED_QCAP,
                    [=](uint32_t sym, int t, uint32_t word) {
                        if (t == 1 && !has2) return;
                        const uint32_t e = sym + 1u;
                        uint32_t *wp = base + ((t ? gstride : 0u) + (e / 32u) * 32u);
                        const uint32_t bit = 1u << (e & 31u);
                        while (word) {
                            const int l = __ffs(word) - 1;
                            word &= word - 1;
                            atomicOr(wp + l, bit);
                        }
                    });
}

sp_status launch_draw_dense(const sp_program *P, uint64_t seed, uint64_t shot0, int64_t ngroups, uint32_t *Bd,
                            int64_t bpitch, cudaStream_t s)
{
    if (ngroups == 0) return SP_OK;
    const int64_t nvec = ngroups * bpitch * 8;
    k_dense_fill<<<(unsigned)ceil_div(nvec, 256), 256, 0, s>>>(Bd, bpitch, nvec);
    SP_CUDA(cudaGetLastError());
    if (P->n_blk == 0) return SP_OK;
    // a warp's queued events address the blocks of its range (at most all)
    if ((uint64_t)P->n_blk >= event_max_blocks(2))
        return set_error(SP_ERR_INVALID_ARG, "too many channel blocks for the dense draw");
    // split the channel blocks so that about four waves of warps run (4
    // CTAs of 8 warps per SM), each range keeping at least 64 groups
    const int64_t ctas = ceil_div(ceil_div(ngroups, 2), 8);
    const int64_t want = 4 * 4 * (int64_t)std::max(P->num_sms, 1);
    const int64_t ngrp = ceil_div(P->n_blk, (int64_t)DRAW_GROUP);
    const int64_t ranges = std::max<int64_t>(1, std::min<int64_t>({ceil_div(want, ctas), ngrp / 64, 65535}));
    if ((uint64_t)bpitch * 64u >= (1ull << 32)) return set_error(SP_ERR_INVALID_ARG, "shots too wide for the dense draw");
    // the round keys as launch parameters, and the launch's block constants
    // when all its shots share a high word (as for the push draw)
    Keys K;
    for (int r = 0; r < 10; r++) {
        K.k0[r] = (uint32_t)seed + (uint32_t)r * PH_W0;
        K.k1[r] = (uint32_t)(seed >> 32) + (uint32_t)r * PH_W1;
    }
    const uint4 *consts = nullptr;
    if (P->d_blkConst && (shot0 >> 32) == ((shot0 + 32u * (uint64_t)ngroups - 1u) >> 32)) {
        k_block_consts<<<(unsigned)ceil_div(P->n_blk, 256), 256, 0, s>>>(P->n_blk, (uint32_t)seed,
                                                                        (uint32_t)(shot0 >> 32), P->d_blkFilt,
                                                                        P->d_blkConst);
        SP_CUDA(cudaGetLastError());
        consts = P->d_blkConst;
    }
    k_draw_dense<<<dim3((unsigned)ctas, (unsigned)ranges), 256, 0, s>>>(P->d_blkT, P->d_blkMeta, P->d_blkSym0,
                                                                        P->d_blkFilt, consts, P->n_blk, seed, K,
                                                                        shot0, ngroups, Bd, bpitch);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {
template <typename T>
sp_status upload(T **dst, const std::vector<T> &src, cudaStream_t s)
{
    const size_t n = std::max<size_t>(src.size(), 1);
    if (dev_alloc((void **)dst, n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *dst = nullptr;
        return set_error(SP_ERR_OOM, "cudaMalloc of the sampler program failed");
    }
    if (!src.empty()) SP_CUDA(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return SP_OK;
}

// Longest-processing-time assignment: items (already sorted by decreasing
// cost) go one by one to the least loaded of nt threads.
double lpt_assign(const std::vector<int64_t> &items, const std::vector<double> &cost, int nt, std::vector<int32_t> &owner)
{
    std::vector<std::pair<double, int>> heap;
    for (int t = 0; t < nt; t++) heap.push_back({0.0, t});
    auto cmp = [](const std::pair<double, int> &a, const std::pair<double, int> &b) {
        return a.first > b.first || (a.first == b.first && a.second > b.second);
    };
    std::make_heap(heap.begin(), heap.end(), cmp);
    double mx = 0.0;
    for (int64_t it : items) {
        std::pop_heap(heap.begin(), heap.end(), cmp);
        auto h = heap.back();
        heap.pop_back();
        owner[it] = h.second;
        h.first += cost[it];
        mx = std::max(mx, h.first);
        heap.push_back(h);
        std::push_heap(heap.begin(), heap.end(), cmp);
    }
    return mx;
}
}  // namespace

static uint32_t aux_offset(const sp_program *P, int tw);
size_t fused_words(const sp_program *P, int tw);

sp_status build_fused_program(sp_program *P, cudaStream_t s)
{
    // ---- channel-block draw descriptors ---------------------------------
    const int64_t nch = P->n_ch;
    std::vector<uint32_t> T((size_t)nch);
    std::vector<uint8_t> kind((size_t)nch);
    if (nch) {
        SP_CUDA(cudaMemcpyAsync(T.data(), P->d_chT, (size_t)nch * 4, cudaMemcpyDeviceToHost, s));
        SP_CUDA(cudaMemcpyAsync(kind.data(), P->d_chKind, (size_t)nch, cudaMemcpyDeviceToHost, s));
        SP_CUDA(cudaStreamSynchronize(s));
    }
    const int64_t nb = (nch + 3) / 4;
    P->n_blk = nb;
    std::vector<uint4> bT((size_t)nb);
    std::vector<uint32_t> bMeta((size_t)nb), bSym0((size_t)nb + 1, 0), bFilt((size_t)nb + 1, 0);
    uint32_t sym = 0;
    for (int64_t b = 0; b < nb; b++) {
        uint32_t Tv[4] = {0, 0, 0, 0}, meta = 0, off = 0;
        bSym0[b] = sym;
        for (int i = 0; i < 4; i++) {
            const int64_t c = 4 * b + i;
            if (c >= nch) continue;
            const uint32_t kd = kind[c] == CK_DEP1 ? CK_DEP1 : kind[c] == CK_DEP2 ? CK_DEP2 : CK_BERN;
            const uint32_t k = kd == CK_DEP2 ? 4u : kd == CK_DEP1 ? 2u : 1u;
            Tv[i] = T[c];
            meta |= kd << (2 * i);
            meta |= off << (8 + 4 * i);
            off += k;
        }
        meta |= off << 24;
        bT[b] = make_uint4(Tv[0], Tv[1], Tv[2], Tv[3]);
        bMeta[b] = meta;
        sym += off;
    }
    bSym0[nb] = sym;
    if ((int64_t)sym != P->n_sym) return set_error(SP_ERR_CUDA, "channel symbol count mismatch");
    sp_status st;

    // ---- product program: the measurement rows' own parts by symbol -------
    const int64_t R = P->n_rows;
    const int64_t M = P->n_meas;
    std::vector<int32_t> parent((size_t)R);
    std::vector<uint8_t> cflag((size_t)R);
    std::vector<uint32_t> off((size_t)R + 1);
    if (R) {
        SP_CUDA(cudaMemcpyAsync(parent.data(), P->d_parent, (size_t)R * 4, cudaMemcpyDeviceToHost, s));
        SP_CUDA(cudaMemcpyAsync(cflag.data(), P->d_cflag, (size_t)R, cudaMemcpyDeviceToHost, s));
        SP_CUDA(cudaMemcpyAsync(off.data(), P->d_rowOff, ((size_t)R + 1) * 4, cudaMemcpyDeviceToHost, s));
        SP_CUDA(cudaStreamSynchronize(s));
    }
    std::vector<uint32_t> own_idx(R ? (size_t)off[M] : 0u);
    if (!own_idx.empty())
        SP_CUDA(cudaMemcpy(own_idx.data(), P->d_idx, own_idx.size() * 4, cudaMemcpyDeviceToHost));
    for (int64_t j = 0; j < M; j++)
        if (parent[j] >= M) return set_error(SP_ERR_CUDA, "measurement row with a non-measurement parent");
    // transpose row -> symbols (the own parts) into symbol -> rows
    std::vector<uint32_t> colOff((size_t)P->n_sym + 1, 0), colRows(own_idx.size());
    for (uint32_t v : own_idx) {
        if ((int64_t)v >= P->n_sym) return set_error(SP_ERR_CUDA, "own-part symbol out of range");
        colOff[v + 1]++;
    }
    for (int64_t v = 0; v < P->n_sym; v++) colOff[v + 1] += colOff[v];
    {
        std::vector<uint32_t> pos(colOff.begin(), colOff.end() - 1);
        for (int64_t j = 0; j < M; j++)
            for (uint32_t k = off[j]; k < off[j + 1]; k++) colRows[pos[own_idx[k]]++] = (uint32_t)j;
    }
    if ((st = upload(&P->d_colOff, colOff, s)) || (st = upload(&P->d_colRows, colRows, s))) return st;
    // A channel none of whose symbols is held by a measurement row's own
    // part changes no record (every record row is an XOR of own parts along
    // a parent chain, and detectors and observables are XORs of measurement
    // rows), so the sampler's copy of its threshold is zero and its block is
    // skipped by the draws when no channel of it can fire.  The channel
    // table keeps the circuit's thresholds.
    int64_t live_blocks = 0;
    for (int64_t b = 0; b < nb; b++) {
        uint32_t Tv[4] = {bT[b].x, bT[b].y, bT[b].z, bT[b].w};
        const uint32_t meta = bMeta[b];
        for (int i = 0; i < 4; i++) {
            if (4 * b + i >= nch) continue;
            const uint32_t kd = (meta >> (2 * i)) & 3u;
            const uint32_t k = kd == CK_DEP2 ? 4u : kd == CK_DEP1 ? 2u : 1u;
            const uint32_t v0 = bSym0[b] + ((meta >> (8 + 4 * i)) & 15u);
            bool held = false;
            for (uint32_t v = v0; v < v0 + k; v++) held = held || colOff[v + 1] > colOff[v];
            if (!held) Tv[i] = 0u;
        }
        bT[b] = make_uint4(Tv[0], Tv[1], Tv[2], Tv[3]);
        const uint64_t sumT = (uint64_t)Tv[0] + Tv[1] + Tv[2] + Tv[3];
        bFilt[b] = sumT >= FREQUENT_SUM ? FREQUENT : std::max(std::max(Tv[0], Tv[1]), std::max(Tv[2], Tv[3]));
        live_blocks += bFilt[b] != 0u;
    }
    P->n_blk_live = live_blocks;
    if ((st = upload(&P->d_blkT, bT, s)) || (st = upload(&P->d_blkMeta, bMeta, s)) || (st = upload(&P->d_blkSym0, bSym0, s)) ||
        (st = upload(&P->d_blkFilt, bFilt, s)))
        return st;
    if (dev_alloc((void **)&P->d_blkConst, (size_t)std::max<int64_t>(nb, 1) * sizeof(uint4)) != cudaSuccess) {
        cudaGetLastError();
        P->d_blkConst = nullptr;
        return set_error(SP_ERR_OOM, "cudaMalloc of the block constants failed");
    }
    // step 0: constants of the own parts
    std::vector<uint8_t> cf(cflag.begin(), cflag.begin() + M);
    // step B: parent chains, whole trees per thread, parents first
    const int NT = FUSED_THREADS;
    std::vector<int64_t> root((size_t)M);
    std::vector<double> tsize((size_t)M, 0.0);
    for (int64_t j = 0; j < M; j++) {
        root[j] = parent[j] >= 0 ? root[parent[j]] : j;
        if (parent[j] >= 0) tsize[root[j]] += 1.0;
    }
    std::vector<int64_t> trees;
    for (int64_t j = 0; j < M; j++) if (root[j] == j && tsize[j] > 0) trees.push_back(j);
    std::stable_sort(trees.begin(), trees.end(), [&](int64_t a, int64_t b) { return tsize[a] > tsize[b]; });
    std::vector<int32_t> ownerT((size_t)M, 0);
    lpt_assign(trees, tsize, NT, ownerT);
    std::vector<uint32_t> bOff((size_t)NT + 1, 0);
    for (int64_t j = 0; j < M; j++) if (parent[j] >= 0) bOff[ownerT[root[j]] + 1]++;
    for (int t = 0; t < NT; t++) bOff[t + 1] += bOff[t];
    std::vector<uint2> bItem((size_t)bOff[NT]);
    {
        std::vector<uint32_t> pos(bOff.begin(), bOff.end() - 1);
        for (int64_t j = 0; j < M; j++)   // increasing j: parents before children
            if (parent[j] >= 0) bItem[pos[ownerT[root[j]]]++] = make_uint2((uint32_t)j, (uint32_t)parent[j]);
    }
    P->fused_items = (int64_t)bItem.size();
    if ((st = upload(&P->d_fCflag, cf, s)) || (st = upload(&P->d_fChain, bItem, s)) || (st = upload(&P->d_fBOff, bOff, s)) ||
        (st = upload(&P->d_fCOff, P->h_xoff, s)) || (st = upload(&P->d_fCRefs, P->h_xrefs, s)))
        return st;

    // ---- default variant: the records of a tile must fit in shared memory --
    int dev = 0, smem_max = 0, nsm = 0;
    SP_CUDA(cudaGetDevice(&dev));
    SP_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    SP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    P->num_sms = nsm;
    P->smem_max = smem_max;
    P->fused_tw = 0;
    // queued events address blocks relative to a warp's first block
    const bool events_ok = (uint64_t)nb / (FUSED_THREADS / 32) + 1 < event_max_blocks(2);
    if (R > 0 && nb > 0 && events_ok) {
        if (fused_words(P, 2) * 4 <= (size_t)smem_max) st = fused_select(P, 2, 1);
        else if (fused_words(P, 1) * 4 <= (size_t)smem_max) st = fused_select(P, 1, 1);
        if (st != SP_OK) return st;
    }
    return SP_OK;
}

static uint32_t aux_offset(const sp_program *P, int tw) { return (uint32_t)((P->n_rows * tw + 3) / 4 * 4); }

// Words of the phase-2 tables when staged in shared memory (a multiple of 4).
static size_t table_words(const sp_program *P)
{
    const size_t w = 2 * (size_t)P->fused_items + (FUSED_THREADS + 1) + (size_t)(P->n_det + P->n_obs + 1) +
                     (size_t)P->h_xrefs.size();
    return (w + 3) / 4 * 4;
}

// Shared-memory words of a tile of 32*tw shots: the records R_s (n_rows x tw
// words), then a region used by the warps' event queues in phase 1 and by
// the emit stage in phase 3 (one record kind at a time, or all three side
// by side when emit_once).
size_t fused_words(const sp_program *P, int tw, bool emit_once)
{
    int64_t max_words = 0, sum_words = 0;
    for (int64_t n : {P->n_meas, P->n_det, P->n_obs}) {
        max_words = std::max<int64_t>(max_words, 2 * ((n + 63) / 64) + 1);
        sum_words += 2 * ((n + 63) / 64) + 1;
    }
    const int64_t stage_words = 32 * tw * (emit_once ? sum_words : max_words);
    const int64_t queue_words = (FUSED_THREADS / 32) * (int64_t)FUSED_QCAP;
    return (size_t)aux_offset(P, tw) + (size_t)std::max(stage_words, queue_words);
}

size_t fused_words(const sp_program *P, int tw) { return fused_words(P, tw, false); }

typedef void (*FusedFn)(FusedParams);

static FusedFn fused_kernel(int tw, int unroll)
{
    if (tw == 4) return unroll == 2 ? k_fused<4, 2> : k_fused<4, 1>;
    if (tw == 2) return unroll == 3 ? k_fused<2, 3> : unroll == 2 ? k_fused<2, 2> : k_fused<2, 1>;
    return unroll == 2 ? k_fused<1, 2> : k_fused<1, 1>;
}

sp_status fused_select(sp_program *P, int tw, int unroll)
{
    if ((tw != 1 && tw != 2 && tw != 4) || unroll < 1 || unroll > 3 || (unroll == 3 && tw != 2))
        return set_error(SP_ERR_INVALID_ARG, "tile words must be 1, 2 or 4, variant 1 or 2 (3: 64-shot tiles only)");
    if (P->n_rows == 0 || P->n_blk == 0) return set_error(SP_ERR_INVALID_ARG, "nothing to sample on the fused path");
    const int threads = fused_threads(tw, unroll);
    if ((uint64_t)P->n_blk / (uint64_t)(threads / 32) + 1 >= event_max_blocks(tw))
        return set_error(SP_ERR_INVALID_ARG, "too many channel blocks for the fused path");
    const size_t bytes = fused_words(P, tw) * 4;
    if (bytes > (size_t)P->smem_max)
        return set_error(SP_ERR_INVALID_ARG, "the records of that fused tile do not fit in shared memory");
    FusedFn fn = fused_kernel(tw, unroll);
    // The limit is a property of the kernel, shared by every program: keep it
    // at the device maximum so that no program's choice lowers another's.
    SP_CUDA(max_dynamic_smem(fn));
    int occ = 0;
    SP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, bytes));
    // the one-pass emit and the phase-2 tables in shared memory, each where
    // it keeps the CTAs per SM of the plain layout (both, else the emit, else
    // the tables)
    struct Opt { bool once, tab; };
    Opt pick{false, false};
    size_t pick_bytes = bytes;
    int pick_occ = occ;
    for (Opt o : {Opt{true, true}, Opt{true, false}, Opt{false, true}}) {
        const size_t b = (fused_words(P, tw, o.once) + (o.tab ? table_words(P) : 0)) * 4;
        if (b > (size_t)P->smem_max) continue;
        int oc = 0;
        SP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oc, fn, threads, b));
        if (oc >= occ && oc > 0) {
            pick = o;
            pick_bytes = b;
            pick_occ = oc;
            break;
        }
    }
    P->fused_tw = tw;
    P->fused_unroll = unroll;
    P->fused_threads = threads;
    P->fused_smem_base = bytes;
    P->fused_smem = pick_bytes;
    P->fused_emit_once = pick.once;
    P->fused_tab_off = pick.tab ? (uint32_t)fused_words(P, tw, pick.once) : 0u;
    P->fused_aux_off = aux_offset(P, tw);
    P->fused_ctas_per_sm = std::max(pick_occ, 1);
    return SP_OK;
}

// Autotuner: time the fused variants that fit -- 64-shot tiles at two CTAs
// per SM, 32-shot tiles, 64-shot tiles at one CTA per SM with more registers,
// 128-shot tiles at 256 threads x two CTAs or 512 threads x one CTA per SM --
// on a few tiles per SM, drawing with the program's current fault-draw
// stream, and keep the fastest.  The choice is cached per circuit shape and
// stream for the process.
sp_status autotune(sp_program *P, cudaStream_t s)
{
    if (!P->fused_tw) return SP_OK;
    typedef std::tuple<int, int64_t, int64_t, int64_t, int64_t, int64_t, int> Key;
    static std::mutex mu;
    static std::map<Key, std::pair<int, int>> cache;
    const Key key{P->device, P->n_sym, P->n_rows, P->n_blk, P->nnz_delta, P->n_meas, P->stream};
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            P->tuned = true;
            return fused_select(P, it->second.first, it->second.second);
        }
    }
    int smem_sm = 0;
    SP_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, P->device));
    std::vector<std::pair<int, int>> cand;
    for (auto c : {std::make_pair(2, 1), std::make_pair(1, 1), std::make_pair(2, 2), std::make_pair(2, 3),
                   std::make_pair(4, 1), std::make_pair(4, 2)}) {
        const size_t bytes = fused_words(P, c.first) * 4;
        if (bytes > (size_t)P->smem_max) continue;
        // the 4-CTA shape only where four tiles' records fit in one SM
        if (c.second == 3 && 4 * (bytes + 1024) > (size_t)smem_sm) continue;
        cand.push_back(c);
    }
    const uint64_t shots = (uint64_t)P->num_sms * 2u * 64u * 4u;
    const int64_t wm = (P->n_meas + 63) / 64, wd = (P->n_det + 63) / 64, wo = (P->n_obs + 63) / 64;
    uint64_t *out = nullptr;
    if (dev_alloc((void **)&out, (size_t)shots * (size_t)std::max<int64_t>(wm + wd + wo, 1) * 8) != cudaSuccess) {
        cudaGetLastError();
        return set_error(SP_ERR_OOM, "cudaMalloc of the autotuner outputs failed");
    }
    uint64_t *om = out, *od = out + shots * wm, *oo = od + shots * wd;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    std::pair<int, int> pick(P->fused_tw, P->fused_unroll);
    sp_status st = SP_OK;
    const bool prof = P->profiling;
    P->profiling = false;
    // candidates are timed twice (best of two); another variant replaces the
    // default (the first candidate) only when it is at least 3% faster, so
    // timing noise does not flip the choice between equivalent variants
    for (size_t ci = 0; ci < cand.size(); ci++) {
        const auto &c = cand[ci];
        if ((st = fused_select(P, c.first, c.second)) != SP_OK) break;
        if ((st = fused_chunk(P, 1, 0, shots, om, od, oo, s)) != SP_OK) break;
        P->autotune_launches += 1;
        float ms = 1e30f;
        for (int rep = 0; rep < 2 && st == SP_OK; rep++) {
            cudaEventRecord(e0, s);
            st = fused_chunk(P, 1, shots * (rep + 1), shots, om, od, oo, s);
            cudaEventRecord(e1, s);
            P->autotune_launches += 1;
            if (cudaEventSynchronize(e1) != cudaSuccess) { st = cuda_error(cudaGetLastError(), "autotune"); break; }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            ms = std::min(ms, t);
        }
        if (st != SP_OK) break;
        if (ci == 0 || ms < 0.97f * best) { best = ms; pick = c; }
    }
    P->profiling = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dev_free(out);
    if (st != SP_OK) return st;
    {
        std::lock_guard<std::mutex> lock(mu);
        cache[key] = pick;
    }
    P->tuned = true;
    return fused_select(P, pick.first, pick.second);
}

sp_status launch_draw_staged(const sp_program *P, uint64_t seed, uint64_t shot0, int64_t nwords, uint32_t *B,
                             int64_t pitch, cudaStream_t s)
{
    if (P->n_sym == 0 || nwords == 0) return SP_OK;
    // about four waves of warps, each range keeping at least 256 channel blocks
    const int64_t want = 4 * 32 * (int64_t)std::max(P->num_sms, 1);
    const int64_t ranges = std::max<int64_t>(1, std::min<int64_t>({ceil_div(want, nwords), P->n_blk / 256, 65535}));
    k_draw_staged<<<dim3((unsigned)ceil_div(nwords, 8), (unsigned)ranges), 256, 0, s>>>(
        P->d_blkT, P->d_blkMeta, P->d_blkSym0, P->n_blk, P->n_sym, seed, shot0, nwords, B, pitch);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

FusedParams fused_params(const sp_program *P, int tw, uint64_t seed, uint64_t shot0, uint64_t nshots,
                         uint64_t *d_meas, uint64_t *d_det, uint64_t *d_obs)
{
    FusedParams fp;
    memset(&fp, 0, sizeof fp);
    fp.blkT = P->d_blkT; fp.blkMeta = P->d_blkMeta; fp.blkSym0 = P->d_blkSym0; fp.blkFilt = P->d_blkFilt;
    fp.colOff = P->d_colOff; fp.colRows = P->d_colRows;
    fp.n_blk = P->n_blk; fp.n_rows = P->n_rows; fp.n_meas = P->n_meas; fp.n_det = P->n_det; fp.n_obs = P->n_obs;
    fp.cflag = P->d_fCflag; fp.bItem = P->d_fChain; fp.bOff = P->d_fBOff;
    fp.cOff = P->d_fCOff; fp.cRefs = P->d_fCRefs;
    fp.seed = seed; fp.shot0 = shot0; fp.nshots = nshots;
    fp.out[0] = d_meas; fp.out[1] = d_det; fp.out[2] = d_obs;
    fp.rows0[0] = 0; fp.rows0[1] = P->n_meas; fp.rows0[2] = P->n_meas + P->n_det;
    fp.nrow[0] = P->n_meas; fp.nrow[1] = P->n_det; fp.nrow[2] = P->n_obs;
    fp.aux_off_words = aux_offset(P, tw);
    for (int r = 0; r < 10; r++) {
        fp.keys.k0[r] = (uint32_t)seed + (uint32_t)r * PH_W0;
        fp.keys.k1[r] = (uint32_t)(seed >> 32) + (uint32_t)r * PH_W1;
    }
    fp.s2Ch = P->d_s2Ch; fp.s2G = P->d_s2G; fp.s2Rand = P->d_s2Rand;
    fp.n_fault = (uint32_t)P->s2_nfault; fp.n_grp = (uint32_t)P->s2_ngrp; fp.n_rnd = (uint32_t)P->s2_nrnd;
    fp.tab_off_words = tw == P->fused_tw ? P->fused_tab_off : 0u;
    fp.emit_once = tw == P->fused_tw && P->fused_emit_once ? 1u : 0u;
    fp.n_items = (uint32_t)P->fused_items;
    fp.n_refs = (uint32_t)P->h_xrefs.size();
    return fp;
}

sp_status fused_chunk(sp_program *P, uint64_t seed, uint64_t shot0, uint64_t nshots, uint64_t *d_meas,
                      uint64_t *d_det, uint64_t *d_obs, cudaStream_t s)
{
    if (nshots == 0) return SP_OK;
    if (!P->fused_tw) return set_error(SP_ERR_INVALID_ARG, "fused path unavailable for this program");
    if (P->stream == 2) return grouped_chunk(P, seed, shot0, nshots, d_meas, d_det, d_obs, s);
    FusedParams fp = fused_params(P, P->fused_tw, seed, shot0, nshots, d_meas, d_det, d_obs);
    // one launch's block constants when its shots share a high word and it
    // runs at least two waves of tiles (a short launch would pay the extra
    // kernel's latency for little)
    const uint64_t wave = 32u * (uint64_t)P->fused_tw * (uint64_t)P->num_sms * (uint64_t)P->fused_ctas_per_sm;
    if (P->d_blkConst && nshots >= 2 * wave && (shot0 >> 32) == ((shot0 + nshots - 1) >> 32)) {
        ProfScope pc(P, SP_KERNEL_CONSTS, s);
        k_block_consts<<<(unsigned)ceil_div(P->n_blk, 256), 256, 0, s>>>(P->n_blk, (uint32_t)seed,
                                                                        (uint32_t)(shot0 >> 32), P->d_blkFilt,
                                                                        P->d_blkConst);
        SP_CUDA(cudaGetLastError());
        fp.blkConst = P->d_blkConst;
    }
    const uint64_t per_tile = 32u * (uint64_t)P->fused_tw;
    const uint64_t ntiles = (nshots + per_tile - 1) / per_tile;
    const uint64_t grid = std::min<uint64_t>(ntiles, (uint64_t)P->num_sms * (uint64_t)P->fused_ctas_per_sm);
    ProfScope ps(P, SP_KERNEL_FUSED, s);
    FusedFn fn = fused_kernel(P->fused_tw, P->fused_unroll);
    fn<<<dim3((unsigned)grid), dim3((unsigned)P->fused_threads), P->fused_smem, s>>>(fp);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

// ---------------------------------------------------------------------------
// Batched sampling: plan, capture, replay
// ---------------------------------------------------------------------------
// A plan belongs to one (device, program set, configuration generations,
// shot counts).  It holds, per launch shape, the members' FusedParams in
// device memory, their tile ends and a work counter, and a CUDA graph that
// zeroes the counters and runs one persistent k_fused_batch per shape.  The
// graph reads seeds and output pointers from the parameter block, which
// every call refreshes with one copy on the caller's stream before it
// launches the graph, so new seeds or buffers reuse the plan.  The graph
// touches only build-time tables of its programs (no per-program scratch),
// and a program's plans are dropped when it is freed or reconfigured.
// Members without a fused kernel (or set to another path) are sampled
// through their own path on the caller's stream after the graph.
namespace {

typedef void (*BatchFn)(const FusedParams *, int, const uint64_t *, unsigned long long *);

BatchFn batch_kernel(int tw, int unroll)
{
    if (tw == 4) return unroll == 2 ? k_fused_batch<4, 2> : k_fused_batch<4, 1>;
    if (tw == 2) return unroll == 3 ? k_fused_batch<2, 3> : unroll == 2 ? k_fused_batch<2, 2> : k_fused_batch<2, 1>;
    return unroll == 2 ? k_fused_batch<1, 2> : k_fused_batch<1, 1>;
}

struct BatchGroup {
    int tw = 0, unroll = 0, threads = 0, ctas = 0;
    size_t smem = 0;
    int grid = 0;
    std::vector<uint32_t> members;   // indices into the call's arrays, by decreasing cost per tile
    size_t param0 = 0;               // first entry of this group in the parameter block
};


// A member with at least one full wave of tiles runs as its own k_fused
// node (its launch shape, launch-constant node, staged tables); the graph's
// branches of such nodes fill each other's last waves.
struct SoloMember {
    uint32_t member = 0;
    int grid = 0;
    bool consts = false;                       // a k_block_consts node precedes the kernel
    cudaGraphNode_t consts_node = nullptr, fused_node = nullptr;
};

struct BatchPlan {
    int device = 0;
    std::vector<uint64_t> key;
    std::vector<const sp_program *> progs;
    std::vector<BatchGroup> groups;
    std::vector<SoloMember> solo;
    std::vector<uint32_t> others;              // members sampled through their own path
    size_t nparams = 0;
    FusedParams *d_params = nullptr;           // [nparams], refreshed by every call
    uint64_t *d_tileEnd = nullptr;             // [nparams]
    uint64_t *d_blkEnd = nullptr;              // [nparams] cumulative channel blocks, parameter order
    uint64_t nblk_total = 0;
    unsigned long long *d_counter = nullptr;   // [groups]
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t last_use = 0;
    ~BatchPlan()
    {
        // launches of this plan may still be in flight
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != device) cudaSetDevice(device);
        cudaDeviceSynchronize();
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        dev_free(d_params);
        dev_free(d_tileEnd);
        dev_free(d_blkEnd);
        dev_free(d_counter);
        if (cur >= 0 && cur != device) cudaSetDevice(cur);
        cudaGetLastError();
    }
};

std::mutex g_batch_mu;
std::vector<BatchPlan *> g_plans;
uint64_t g_batch_clock = 0;
// per device: the capture stream and one branch stream per launch shape
constexpr int MAX_SHAPES = 8;
cudaStream_t g_capture_stream[64][MAX_SHAPES] = {};
cudaEvent_t g_capture_event[64][MAX_SHAPES + 1] = {};

// The per-call part of the members' parameters: seeds and output pointers.
// A member's launch constants live in its program's buffer, written by the
// plan's first node; a program that appears more than once in the call
// (its members would share the buffer with different seeds), or a member
// whose shots cross a multiple of 2^32 (the constants hold one high word),
// draws without them.
void fill_params(const BatchPlan &plan, sp_program *const *progs, const uint64_t *seeds, const uint64_t *nshots,
                 uint64_t *const *d_meas, uint64_t *const *d_det, uint64_t *const *d_obs,
                 std::vector<FusedParams> &out)
{
    out.resize(plan.nparams);
    std::map<const sp_program *, int> uses;
    for (const sp_program *P : plan.progs) uses[P]++;
    for (const BatchGroup &g : plan.groups)
        for (size_t k = 0; k < g.members.size(); k++) {
            const uint32_t i = g.members[k];
            out[g.param0 + k] = fused_params(progs[i], g.tw, seeds[i], 0, nshots[i], d_meas ? d_meas[i] : nullptr,
                                             d_det ? d_det[i] : nullptr, d_obs ? d_obs[i] : nullptr);
            out[g.param0 + k].tab_off_words = 0;   // the batch reads phase-2 tables from global memory
            out[g.param0 + k].emit_once = 0;       // and emits one record kind per pass
            const bool own = uses[progs[i]] == 1 && nshots[i] <= (1ull << 32);
            out[g.param0 + k].blkConst = own ? progs[i]->d_blkConst : nullptr;
        }
}

}  // namespace

size_t batch_plan_count()
{
    std::lock_guard<std::mutex> lock(g_batch_mu);
    return g_plans.size();
}

void batch_forget(const sp_program *P)
{
    std::vector<BatchPlan *> drop;
    {
        std::lock_guard<std::mutex> lock(g_batch_mu);
        for (size_t i = 0; i < g_plans.size();) {
            BatchPlan *b = g_plans[i];
            if (std::find(b->progs.begin(), b->progs.end(), P) != b->progs.end()) {
                drop.push_back(b);
                g_plans.erase(g_plans.begin() + i);
            } else {
                i++;
            }
        }
    }
    for (BatchPlan *b : drop) delete b;
}

sp_status sample_batch(sp_program *const *progs, uint32_t n, const uint64_t *seeds, const uint64_t *nshots,
                       uint64_t *const *d_meas, uint64_t *const *d_det, uint64_t *const *d_obs, cudaStream_t s)
{
    int dev = 0;
    SP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(SP_ERR_INVALID_ARG, "device ordinal out of range");
    std::vector<uint64_t> key;
    key.push_back((uint64_t)dev);
    for (uint32_t i = 0; i < n; i++) {
        if (progs[i]->device != dev) return set_error(SP_ERR_INVALID_ARG, "all programs must live on the current device");
        key.insert(key.end(), {(uint64_t)(uintptr_t)progs[i], progs[i]->gen, nshots[i]});
    }
    std::vector<FusedParams> hp;
    std::unique_lock<std::mutex> lock(g_batch_mu);
    BatchPlan *plan = nullptr;
    for (BatchPlan *b : g_plans)
        if (b->key == key) { plan = b; break; }
    if (!plan) {
        // ---- new plan ------------------------------------------------------
        std::unique_ptr<BatchPlan> np(new BatchPlan());
        np->device = dev;
        np->key = key;
        std::map<std::tuple<int, int, int>, BatchGroup> by_shape;
        for (uint32_t i = 0; i < n; i++) {
            const sp_program *P = progs[i];
            np->progs.push_back(P);
            if (nshots[i] == 0) continue;
            if (P->path == SP_PATH_FUSED && P->fused_tw && P->stream == 1) {
                const uint64_t tiles = (nshots[i] + 32u * P->fused_tw - 1) / (32u * P->fused_tw);
                const uint64_t slots = (uint64_t)P->num_sms * (uint64_t)P->fused_ctas_per_sm;
                if (slots && tiles >= slots) {
                    SoloMember m;
                    m.member = i;
                    m.grid = (int)slots;
                    m.consts = P->d_blkConst && tiles >= 2 * slots && nshots[i] <= (1ull << 32) &&
                               std::count(progs, progs + n, progs[i]) == 1;
                    np->solo.push_back(m);
                    continue;
                }
                BatchGroup &g = by_shape[std::make_tuple(P->fused_tw, P->fused_unroll, P->fused_ctas_per_sm)];
                g.tw = P->fused_tw;
                g.unroll = P->fused_unroll;
                g.threads = P->fused_threads;
                g.ctas = P->fused_ctas_per_sm;
                g.smem = std::max(g.smem, P->fused_smem_base);
                g.members.push_back(i);
            } else {
                np->others.push_back(i);
            }
        }
        std::vector<uint64_t> tileEnd, blkEnd;
        // the group with the most work first: the others' CTAs fill its tail
        std::vector<BatchGroup> shapes;
        for (auto &kv : by_shape) shapes.push_back(kv.second);
        auto work = [&](const BatchGroup &g) {
            double w = 0;
            for (uint32_t i : g.members) w += (double)progs[i]->n_blk * (double)nshots[i];
            return w;
        };
        std::stable_sort(shapes.begin(), shapes.end(),
                         [&](const BatchGroup &a, const BatchGroup &b) { return work(a) > work(b); });
        for (BatchGroup g : shapes) {
            std::stable_sort(g.members.begin(), g.members.end(),
                             [&](uint32_t a, uint32_t b) { return progs[a]->n_blk > progs[b]->n_blk; });
            g.param0 = tileEnd.size();
            uint64_t acc = 0;
            for (uint32_t i : g.members) {
                acc += (nshots[i] + 32u * g.tw - 1) / (32u * g.tw);
                tileEnd.push_back(acc);
                np->nblk_total += (uint64_t)progs[i]->n_blk;
                blkEnd.push_back(np->nblk_total);
            }
            BatchFn fn = batch_kernel(g.tw, g.unroll);
            SP_CUDA(max_dynamic_smem(fn));
            int occ = 0;
            SP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, g.threads, g.smem));
            int nsm = 0;
            SP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
            g.grid = (int)std::min<uint64_t>(acc, (uint64_t)nsm * (uint64_t)std::max(occ, 1));
            np->groups.push_back(g);
        }
        np->nparams = tileEnd.size();
        if (np->nparams) {
            if (dev_alloc((void **)&np->d_params, np->nparams * sizeof(FusedParams)) != cudaSuccess ||
                dev_alloc((void **)&np->d_tileEnd, np->nparams * 8) != cudaSuccess ||
                dev_alloc((void **)&np->d_blkEnd, np->nparams * 8) != cudaSuccess ||
                dev_alloc((void **)&np->d_counter, np->groups.size() * 8) != cudaSuccess) {
                cudaGetLastError();
                return set_error(SP_ERR_OOM, "cudaMalloc of the batch plan failed");
            }
            SP_CUDA(cudaMemcpy(np->d_tileEnd, tileEnd.data(), tileEnd.size() * 8, cudaMemcpyHostToDevice));
            SP_CUDA(cudaMemcpy(np->d_blkEnd, blkEnd.data(), blkEnd.size() * 8, cudaMemcpyHostToDevice));
            // ---- capture on library streams, replay on the caller's --------
            // counter reset, then one branch per launch shape (the shapes'
            // persistent kernels may overlap), then a join
            const size_t ng = np->groups.size();
            if (ng > MAX_SHAPES) return set_error(SP_ERR_INVALID_ARG, "too many launch shapes in one batch");
            for (size_t k = 0; k < ng; k++)
                if (!g_capture_stream[dev][k])
                    SP_CUDA(cudaStreamCreateWithFlags(&g_capture_stream[dev][k], cudaStreamNonBlocking));
            for (size_t k : {(size_t)MAX_SHAPES, (size_t)1, (size_t)2, (size_t)3, (size_t)4, (size_t)5, (size_t)6, (size_t)7})
                if (k == MAX_SHAPES || k < ng)
                    if (!g_capture_event[dev][k])
                        SP_CUDA(cudaEventCreateWithFlags(&g_capture_event[dev][k], cudaEventDisableTiming));
            cudaStream_t cs = g_capture_stream[dev][0];
            SP_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            sp_status st = SP_OK;
            auto ok = [&](cudaError_t e, const char *what) {
                if (e != cudaSuccess && st == SP_OK) st = cuda_error(e, what);
            };
            ok(cudaMemsetAsync(np->d_counter, 0, ng * 8, cs), "counter reset during capture");
            if (np->nblk_total) {
                k_block_consts_batch<<<(unsigned)ceil_div((int64_t)np->nblk_total, 256), 256, 0, cs>>>(
                    np->d_params, (int)np->nparams, np->d_blkEnd);
                ok(cudaGetLastError(), "batch block constants during capture");
            }
            ok(cudaEventRecord(g_capture_event[dev][MAX_SHAPES], cs), "fork during capture");
            for (size_t k = 0; k < ng && st == SP_OK; k++) {
                const BatchGroup &g = np->groups[k];
                cudaStream_t bs = g_capture_stream[dev][k];
                if (k) ok(cudaStreamWaitEvent(bs, g_capture_event[dev][MAX_SHAPES], 0), "fork during capture");
                batch_kernel(g.tw, g.unroll)<<<g.grid, g.threads, g.smem, bs>>>(
                    np->d_params + g.param0, (int)g.members.size(), np->d_tileEnd + g.param0, np->d_counter + k);
                ok(cudaGetLastError(), "batch kernel launch during capture");
                if (k) {
                    ok(cudaEventRecord(g_capture_event[dev][k], bs), "join during capture");
                    ok(cudaStreamWaitEvent(cs, g_capture_event[dev][k], 0), "join during capture");
                }
            }
            cudaGraph_t graph = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
            if (st != SP_OK) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            if (ec != cudaSuccess) return cuda_error(ec, "cudaStreamEndCapture");
            np->graph = graph;
        }
        if (!np->solo.empty()) {
            if (!np->graph) SP_CUDA(cudaGraphCreate(&np->graph, 0));
            // heaviest first, each to the least loaded of up to four branches
            std::stable_sort(np->solo.begin(), np->solo.end(), [&](const SoloMember &a, const SoloMember &b) {
                return (double)progs[a.member]->n_blk * (double)nshots[a.member] >
                       (double)progs[b.member]->n_blk * (double)nshots[b.member];
            });
            const int nb = (int)std::min<size_t>(4, np->solo.size());
            std::vector<double> load((size_t)nb, 0.0);
            std::vector<cudaGraphNode_t> tail((size_t)nb, nullptr);
            for (SoloMember &m : np->solo) {
                const int br = (int)(std::min_element(load.begin(), load.end()) - load.begin());
                load[br] += (double)progs[m.member]->n_blk * (double)nshots[m.member];
                const sp_program *P = progs[m.member];
                // parameters of the first call; every call sets its own
                FusedParams fp = fused_params(P, P->fused_tw, seeds[m.member], 0, nshots[m.member], nullptr,
                                              nullptr, nullptr);
                uint32_t k0 = (uint32_t)seeds[m.member], c1u = 0u;
                int64_t nblk = P->n_blk;
                const uint32_t *filt = P->d_blkFilt;
                uint4 *bconst = P->d_blkConst;
                if (m.consts) {
                    void *args[] = {&nblk, &k0, &c1u, &filt, &bconst};
                    cudaKernelNodeParams kp = {};
                    kp.func = (void *)k_block_consts;
                    kp.gridDim = dim3((unsigned)ceil_div(P->n_blk, 256));
                    kp.blockDim = dim3(256);
                    kp.kernelParams = args;
                    SP_CUDA(cudaGraphAddKernelNode(&m.consts_node, np->graph, tail[br] ? &tail[br] : nullptr,
                                                   tail[br] ? 1 : 0, &kp));
                    tail[br] = m.consts_node;
                    fp.blkConst = P->d_blkConst;
                }
                void *args[] = {&fp};
                cudaKernelNodeParams kp = {};
                kp.func = (void *)fused_kernel(P->fused_tw, P->fused_unroll);
                kp.gridDim = dim3((unsigned)m.grid);
                kp.blockDim = dim3((unsigned)P->fused_threads);
                kp.sharedMemBytes = (unsigned)P->fused_smem;
                kp.kernelParams = args;
                SP_CUDA(cudaGraphAddKernelNode(&m.fused_node, np->graph, tail[br] ? &tail[br] : nullptr,
                                               tail[br] ? 1 : 0, &kp));
                tail[br] = m.fused_node;
            }
        }
        if (np->graph) SP_CUDA(cudaGraphInstantiate(&np->exec, np->graph, 0));
        // bounded cache: drop the least recently used plan
        if (g_plans.size() >= BATCH_MAX_PLANS) {
            auto lru = std::min_element(g_plans.begin(), g_plans.end(),
                                        [](const BatchPlan *a, const BatchPlan *b) { return a->last_use < b->last_use; });
            BatchPlan *old = *lru;
            g_plans.erase(lru);
            delete old;
        }
        plan = np.release();
        g_plans.push_back(plan);
    }
    plan->last_use = ++g_batch_clock;
    if (plan->exec) {
        if (plan->nparams) {
            fill_params(*plan, progs, seeds, nshots, d_meas, d_det, d_obs, hp);
            // pageable source: staged by the runtime before the call returns
            SP_CUDA(cudaMemcpyAsync(plan->d_params, hp.data(), hp.size() * sizeof(FusedParams), cudaMemcpyHostToDevice, s));
        }
        // the solo members' seeds and outputs go into their nodes (a launch
        // already enqueued keeps the parameters it was launched with)
        for (const SoloMember &m : plan->solo) {
            const uint32_t i = m.member;
            const sp_program *P = progs[i];
            FusedParams fp = fused_params(P, P->fused_tw, seeds[i], 0, nshots[i], d_meas ? d_meas[i] : nullptr,
                                          d_det ? d_det[i] : nullptr, d_obs ? d_obs[i] : nullptr);
            if (m.consts) {
                int64_t nblk = P->n_blk;
                uint32_t k0 = (uint32_t)seeds[i], c1u = 0u;
                const uint32_t *filt = P->d_blkFilt;
                uint4 *bconst = P->d_blkConst;
                void *args[] = {&nblk, &k0, &c1u, &filt, &bconst};
                cudaKernelNodeParams kp = {};
                kp.func = (void *)k_block_consts;
                kp.gridDim = dim3((unsigned)ceil_div(P->n_blk, 256));
                kp.blockDim = dim3(256);
                kp.kernelParams = args;
                SP_CUDA(cudaGraphExecKernelNodeSetParams(plan->exec, m.consts_node, &kp));
                fp.blkConst = P->d_blkConst;
            }
            void *args[] = {&fp};
            cudaKernelNodeParams kp = {};
            kp.func = (void *)fused_kernel(P->fused_tw, P->fused_unroll);
            kp.gridDim = dim3((unsigned)m.grid);
            kp.blockDim = dim3((unsigned)P->fused_threads);
            kp.sharedMemBytes = (unsigned)P->fused_smem;
            kp.kernelParams = args;
            SP_CUDA(cudaGraphExecKernelNodeSetParams(plan->exec, m.fused_node, &kp));
        }
        SP_CUDA(cudaGraphLaunch(plan->exec, s));
    }
    const std::vector<uint32_t> others = plan->others;
    lock.unlock();
    for (uint32_t i : others) {
        sp_status st = sample_range(progs[i], seeds[i], 0, nshots[i], d_meas ? d_meas[i] : nullptr,
                                    d_det ? d_det[i] : nullptr, d_obs ? d_obs[i] : nullptr, s);
        if (st != SP_OK) return st;
    }
    return SP_OK;
}

}  // namespace sp
