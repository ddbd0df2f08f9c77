// sp_grouped.cu -- the grouped fault draw (stream 2, opt-in) inside the fused
// sampling kernel.
//
// The draw of b from P_C (Algorithm 1, Sampling) with the same Sec. 3.1
// distributions as the per-channel stream (independent Bernoulli(p) symbols,
// depolarizing outcomes uniform over the non-identity Paulis, random outcomes
// fair coins), drawn with far fewer Philox words when channels rarely fire.
// Counter word 3 tags the words (the per-channel stream uses 0):
//   - random-outcome channel of rank r: bit r%32 of word (r/32)%4 of
//     Philox(shot lo, shot hi, r/128, 3);
//   - the other channels, in channel order, form groups of 32.  Group g
//     fires when word g%4 of Philox(shot lo, shot hi, g/4, 1) is below
//     G_g = floor((1 - prod_i (1 - p_i)) 2^32);
//   - in a group that fired, channel i reads word i%4 of Philox(shot lo,
//     shot hi, 8g + i/4, 2).  While none before it has fired it fires below
//     Q_i = floor(p_i / (1 - prod_{j>=i}(1 - p_j)) 2^32), the last channel
//     with p > 0 always; after the first fired channel each fires below its
//     own T_i = floor(p_i 2^32);
//   - a depolarizing channel that fired takes k = min(floor(u m / U), m - 1),
//     U the threshold that decided it, m = 3 or 15, and symbol s0+i gets bit
//     i of k+1.
// Conditioned on the group firing, the walk picks the first fired channel i
// with probability prod_{j<i}(1 - p_j) p_i / (1 - prod_j (1 - p_j)), and the
// channels after it are independent, so every channel is Bernoulli(p_i),
// independently of the others (up to the 2^-32 quantization of thresholds).
//
// In the kernel, each warp owns a range of groups: per 32-shot word one
// Philox evaluation gives the words of four groups; each (group, shot) that
// fired is queued and walked by one lane (8 Philox blocks of channel words).
// Random outcomes fire in half the shots: a 32x32 transpose turns 32 shots'
// words into one 32-shot column per channel.  Phases 2 and 3 of the tile
// (parent chains, detectors, emit) are those of the per-channel stream.
#include <algorithm>
#include <vector>

#include "sp_fused_dev.cuh"

namespace sp {

constexpr uint32_t S2_GROUP = 32;
constexpr uint32_t S2_TAG_GROUP = 1, S2_TAG_CHANNEL = 2, S2_TAG_RANDOM = 3;
constexpr uint32_t S2_LAST = 4u;   // flag in s2Ch.w: the group's last channel with p > 0

// Philox4x32-10 of counter (shot, ctr2, tag) where s = shot_const(shot,
// k1 ^ tag): round 1's word 2 product depends on the tag through x2.
__device__ __forceinline__ void philox_tagged(const ShotConst &s, uint32_t ctr2, const Keys &K, uint32_t &o0,
                                              uint32_t &o1, uint32_t &o2, uint32_t &o3)
{
    const uint64_t ub = (uint64_t)PH_M1 * ctr2;
    philox_block(s, s.c1, (uint32_t)(ub >> 32), (uint32_t)ub, K, o0, o1, o2, o3);
}

// Symbol bits of a channel decided by threshold U: 1 for a one-symbol
// channel, k+1 with k = min(floor(u m / U), m - 1) for a depolarizing one
// (cat_index is exact for u < U; u >= U happens only for a group's last
// channel with p > 0, which fires regardless, and gives k = m - 1).
__device__ __forceinline__ uint32_t grouped_outcome(uint32_t kind, uint32_t u, uint32_t U)
{
    if (kind != CK_DEP1 && kind != CK_DEP2) return 1u;
    const uint32_t m = kind == CK_DEP1 ? 3u : 15u;
    return (u < U ? cat_index(u, U, m) : m - 1u) + 1u;
}

// Walk the queued (group, shot) events e = lane, lane+32, ... < n; event =
// group - g0 above bit 5 + TB, tile word t, lane.  The loops have the same
// trip counts in every lane (lanes without an event, or past a group's last
// channel, are masked) and the warp reconverges after each block of four
// channel words: a lane leaving a divergent apply loop early would
// otherwise run ahead into the next block's Philox rounds, and the warp
// would execute them in several partial passes.  A lane's walk fires about
// one channel, but some lane of the warp fires in most of the 32 channel
// slots, so the walk only notes (symbol, kind, word, threshold) of its first
// two fired channels, by selects; their outcomes are computed and applied
// after the walk, by every lane at the same point.  A third or later fired
// channel (rare) is applied at once.
template <int TW, typename Apply>
__device__ __forceinline__ void grouped_drain(const uint32_t *q, uint32_t n, const FusedParams &p, const Keys &K,
                                              uint32_t g0, uint64_t shot_base, int lane, const Apply &apply)
{
    __syncwarp();
    constexpr int TB = event_tbits(TW);
    const uint32_t k1 = (uint32_t)(p.seed >> 32);
    for (uint32_t base = 0; base < n; base += 32) {
        const uint32_t e = base + (uint32_t)lane;
        const bool live = e < n;
        const uint32_t ev = live ? q[e] : 0u;
        const uint32_t g = g0 + (ev >> (5 + TB));
        const int t = (ev >> 5) & ((1u << TB) - 1u);
        const uint32_t ln = ev & 31u;
        const ShotConst s = shot_const(shot_base + 32u * (uint32_t)t + ln, k1 ^ S2_TAG_CHANNEL);
        const uint32_t first = g * S2_GROUP;
        const uint32_t nch = live ? min(S2_GROUP, p.n_fault - first) : 0u;
        bool searching = true, have_a = false, have_b = false;
        uint32_t sym_a = 0, w_a = 0, u_a = 0, U_a = 0, sym_b = 0, w_b = 0, u_b = 0, U_b = 0;
        auto apply_bits = [&](uint32_t sym, uint32_t val) {
            while (val) {
                const int b = __ffs(val) - 1;
                val &= val - 1;
                apply(sym + (uint32_t)b, t, 1u << ln);
            }
        };
        // M1 * (8 g + j), the channel block's counter-word product
        uint64_t ub = (uint64_t)PH_M1 * (8u * g);
#pragma unroll 1
        for (uint32_t j = 0; j < S2_GROUP / 4; j++, ub += PH_M1) {
            uint4 c[4];
#pragma unroll
            for (int i = 0; i < 4; i++)
                c[i] = 4 * j + (uint32_t)i < nch ? p.s2Ch[first + 4 * j + (uint32_t)i] : make_uint4(0u, 0u, 0u, 0u);
            uint32_t r[4];
            philox_block(s, s.c1, (uint32_t)(ub >> 32), (uint32_t)ub, K, r[0], r[1], r[2], r[3]);
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const uint32_t u = r[i];
                const uint32_t U = searching ? c[i].x : c[i].y;
                const bool valid = 4 * j + (uint32_t)i < nch;
                const bool fired = valid && (u < U || (searching && (c[i].w & S2_LAST) != 0u));
                const bool to_a = fired && !have_a;
                const bool to_b = fired && have_a && !have_b;
                if (fired && have_b) apply_bits(c[i].z, grouped_outcome(c[i].w & 3u, u, U));
                sym_a = to_a ? c[i].z : sym_a;
                w_a = to_a ? c[i].w : w_a;
                u_a = to_a ? u : u_a;
                U_a = to_a ? U : U_a;
                sym_b = to_b ? c[i].z : sym_b;
                w_b = to_b ? c[i].w : w_b;
                u_b = to_b ? u : u_b;
                U_b = to_b ? U : U_b;
                have_b = have_b || to_b;
                have_a = have_a || fired;
                searching = searching && !fired;
            }
            __syncwarp();
        }
        if (have_a) apply_bits(sym_a, grouped_outcome(w_a & 3u, u_a, U_a));
        if (have_b) apply_bits(sym_b, grouped_outcome(w_b & 3u, u_b, U_b));
        __syncwarp();
    }
    __syncwarp();
}

struct DrawGrouped {
    // phase 1 draws group words: their shot constants carry tag 1
    __device__ static uint32_t shot_key(uint64_t seed) { return (uint32_t)(seed >> 32) ^ S2_TAG_GROUP; }

    template <int TW, typename Apply>
    __device__ static void run(const FusedParams &p, const Keys &K, const Shots<TW> &sc, uint64_t shot_base, int warp,
                               int nwarps, int lane, uint32_t *q, const Apply &apply)
    {
        constexpr int TB = event_tbits(TW);
        const uint32_t k1 = (uint32_t)(p.seed >> 32);
        // ---- random outcomes: 128 channels per Philox block, blocks dealt
        // round robin over the warps
        const uint32_t nrb = (p.n_rnd + 127u) / 128u;
        for (uint32_t rb = (uint32_t)warp; rb < nrb; rb += (uint32_t)nwarps) {
#pragma unroll
            for (int t = 0; t < TW; t++) {
                const ShotConst s = shot_const(shot_base + 32u * (uint32_t)t + (uint32_t)lane, k1 ^ S2_TAG_RANDOM);
                uint32_t w[4];
                philox_tagged(s, rb, K, w[0], w[1], w[2], w[3]);
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    // lane c receives the 32 shots' bits of channel 128 rb + 32 j + c
                    const uint32_t col = transpose32(w[j], lane);
                    const uint32_t r = 128u * rb + 32u * (uint32_t)j + (uint32_t)lane;
                    if (r < p.n_rnd && col) apply(p.s2Rand[r], t, col);
                }
            }
        }
        // ---- the CTA's walk queue: the part of the shared region behind the
        // warps' own queues that phase 3's emit stage uses and phase 1 does
        // not (the same sizes as the host's layout, clamped to the staged
        // tables or the end of the launch's shared memory).  Fired groups
        // go there in sets of 32 and all warps walk them after a barrier,
        // so that the warps that drew more fired groups do not keep the
        // others waiting; what does not fit is walked by its own warp.
        uint32_t *aux = q - warp * (int)FUSED_QCAP;
        uint32_t *cq = aux + nwarps * (int)FUSED_QCAP;
        uint32_t ccap = 0;
        {
            uint32_t mx = 0, sum = 0;
#pragma unroll
            for (int sg = 0; sg < 3; sg++) {
                const uint32_t w = 2u * (uint32_t)((p.nrow[sg] + 63) / 64) + 1u;
                mx = max(mx, w);
                sum += w;
            }
            uint32_t aux_words = max(32u * TW * (p.emit_once ? sum : mx), (FUSED_THREADS / 32) * FUSED_QCAP);
            uint32_t dyn;
            asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
            const uint32_t end = p.tab_off_words ? p.tab_off_words : dyn / 4u;
            aux_words = min(aux_words, end - p.aux_off_words);
            const uint32_t used = (uint32_t)nwarps * FUSED_QCAP + 4u;   // own queues, two counters, padding
            ccap = aux_words > used + 32u ? aux_words - used : 0u;
        }
        uint32_t *cfill = cq, *ctake = cq + 1, *cev = cq + 4;
        if (ccap && threadIdx.x == 0) {
            *cfill = 0u;
            *ctake = 0u;
        }
        __syncthreads();
        // ---- group words: quads [q0, q1) of this warp, 8 quads (32 groups)
        // gathered per queueing step
        const uint32_t nq = (p.n_grp + 3u) / 4u;
        const uint32_t q0 = (uint32_t)((uint64_t)warp * nq / (uint64_t)nwarps);
        const uint32_t q1 = (uint32_t)((uint64_t)(warp + 1) * nq / (uint64_t)nwarps);
        const uint32_t g0 = ccap ? 0u : 4u * q0;   // events hold groups relative to g0
        const uint32_t lt = (1u << lane) - 1u;
        uint32_t cnt = 0;
        // move the first n (<= 32) queued events to the CTA queue; the ones
        // that do not fit stay at the front of the warp's queue (returned)
        auto push = [&](uint32_t n) -> uint32_t {
            __syncwarp();
            uint32_t pos = 0u;
            if (lane == 0) pos = atomicAdd(cfill, n);
            pos = __shfl_sync(FM, pos, 0);
            const uint32_t fit = pos >= ccap ? 0u : min(n, ccap - pos);
            const uint32_t ev = (uint32_t)lane < n ? q[lane] : 0u;
            __syncwarp();
            if ((uint32_t)lane < fit) cev[pos + lane] = ev;
            if ((uint32_t)lane >= fit && (uint32_t)lane < n) q[lane - fit] = ev;
            __syncwarp();
            return n - fit;
        };
        for (uint32_t qq = q0; qq < q1; qq += 8u) {
            const uint32_t nqq = min(8u, q1 - qq);
            uint32_t word[TW];
#pragma unroll
            for (int t = 0; t < TW; t++) word[t] = 0u;
            for (uint32_t k = 0; k < nqq; k++) {
                const uint4 G = p.s2G[qq + k];
#pragma unroll
                for (int t = 0; t < TW; t++) {
                    uint32_t r0, r1, r2, r3;
                    philox_tagged(sc.s[t], qq + k, K, r0, r1, r2, r3);
                    word[t] |= fired4(r0, r1, r2, r3, G) << (4u * k);
                }
            }
            // one event per (group, shot) that fired; a full set of 32 is
            // walked at once
#pragma unroll
            for (int t = 0; t < TW; t++) {
                uint32_t m = word[t];
                while (__any_sync(FM, m != 0u)) {
                    const uint32_t b = m ? (uint32_t)(__ffs(m) - 1) : 0u;
                    const uint32_t bal = __ballot_sync(FM, m != 0u);
                    if (m) q[cnt + __popc(bal & lt)] = ((4u * qq + b - g0) << (5 + TB)) | ((uint32_t)t << 5) | (uint32_t)lane;
                    cnt += __popc(bal);
                    m &= m - 1u;
                    if (cnt >= 32u) {
                        const uint32_t left = ccap ? push(32u) : 32u;
                        if (left) grouped_drain<TW>(q, left, p, K, g0, shot_base, lane, apply);
                        cnt -= 32u;
                        const uint32_t rest = (uint32_t)lane < cnt ? q[32 + lane] : 0u;
                        __syncwarp();
                        if ((uint32_t)lane < cnt) q[lane] = rest;
                        __syncwarp();
                    }
                }
            }
        }
        if (!ccap) {
            grouped_drain<TW>(q, cnt, p, K, g0, shot_base, lane, apply);
            return;
        }
        const uint32_t left = cnt ? push(cnt) : 0u;
        if (left) grouped_drain<TW>(q, left, p, K, g0, shot_base, lane, apply);
        __syncthreads();   // every warp's events are in the CTA queue
        const uint32_t total = min(*cfill, ccap);
        for (;;) {
            uint32_t b = 0u;
            if (lane == 0) b = atomicAdd(ctake, 32u);
            b = __shfl_sync(FM, b, 0);
            if (b >= total) break;
            grouped_drain<TW>(cev + b, min(32u, total - b), p, K, 0u, shot_base, lane, apply);
        }
    }
};

template <int TW, int U>
__global__ void __launch_bounds__(fused_threads(TW, U), fused_minb(TW, U)) k_fused_grouped(FusedParams p)
{
    extern __shared__ __align__(16) uint32_t sm[];
    const uint64_t per_tile = 32u * TW;
    const uint64_t ntiles = (p.nshots + per_tile - 1) / per_tile;
    const FusedTables tab = stage_tables(p, sm);
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
        fused_tile<TW, fused_threads(TW, U), DrawGrouped>(p, p.keys, tab, tile, sm);
}

namespace {
typedef void (*GroupedFn)(FusedParams);

GroupedFn grouped_kernel(int tw, int unroll)
{
    if (tw == 4) return unroll == 2 ? k_fused_grouped<4, 2> : k_fused_grouped<4, 1>;
    if (tw == 2)
        return unroll == 3 ? k_fused_grouped<2, 3> : unroll == 2 ? k_fused_grouped<2, 2> : k_fused_grouped<2, 1>;
    return unroll == 2 ? k_fused_grouped<1, 2> : k_fused_grouped<1, 1>;
}

uint32_t threshold_q(double x)
{
    if (!(x > 0.0)) return 0u;
    const double t = floor(x * 4294967296.0);
    return t >= 4294967295.0 ? 4294967295u : (uint32_t)t;
}

template <typename T>
sp_status upload_vec(T **dst, const std::vector<T> &src, cudaStream_t s)
{
    if (dev_alloc((void **)dst, std::max<size_t>(src.size(), 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *dst = nullptr;
        return set_error(SP_ERR_OOM, "cudaMalloc of the grouped-draw tables failed");
    }
    if (!src.empty()) SP_CUDA(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return SP_OK;
}
}  // namespace

// The grouped draw's tables, from the channels' kinds, first symbols and
// probabilities: per group of 32 channels (random outcomes excluded) its
// threshold G_g; per channel {Q_i, T_i, first symbol, kind | last flag};
// per random outcome its symbol.  Thresholds follow the definition above in
// double precision, channel by channel in order.
sp_status ensure_grouped(sp_program *P, cudaStream_t s)
{
    if (P->d_s2Ch) return SP_OK;
    const int64_t nch = P->n_ch;
    std::vector<uint8_t> kind((size_t)std::max<int64_t>(nch, 1));
    std::vector<uint32_t> sym0((size_t)std::max<int64_t>(nch, 1));
    if (nch) {
        SP_CUDA(cudaMemcpyAsync(kind.data(), P->d_chKind, (size_t)nch, cudaMemcpyDeviceToHost, s));
        SP_CUDA(cudaMemcpyAsync(sym0.data(), P->d_chSym0, (size_t)nch * 4, cudaMemcpyDeviceToHost, s));
        SP_CUDA(cudaStreamSynchronize(s));
    }
    // first symbols as 0-based indices of the symbol -> row lists (channel
    // tables number symbols from 1; symbol 0 is the constant); every symbol
    // a channel sets must exist, checked here before any table is uploaded
    std::vector<int64_t> fault;
    std::vector<uint32_t> rnd;
    for (int64_t c = 0; c < nch; c++) {
        const int64_t ns = kind[c] == CK_DEP2 ? 4 : kind[c] == CK_DEP1 ? 2 : 1;
        if (sym0[c] < 1 || (int64_t)sym0[c] - 1 + ns > P->n_sym)
            return set_error(SP_ERR_CUDA, "channel symbol out of range while building the grouped-draw tables");
        if (kind[c] == CK_RANDOM) rnd.push_back(sym0[c] - 1u);
        else fault.push_back(c);
    }
    if (fault.size() != P->h_fault_p.size())
        return set_error(SP_ERR_CUDA, "channel count mismatch while building the grouped-draw tables");
    const int64_t nf = (int64_t)fault.size();
    const int64_t ngrp = (nf + S2_GROUP - 1) / S2_GROUP;
    std::vector<uint4> ch((size_t)nf), G4((size_t)((ngrp + 3) / 4));
    std::vector<uint32_t> G((size_t)ngrp + 4, 0u);
    for (int64_t g = 0; g < ngrp; g++) {
        const int64_t base = g * S2_GROUP, n = std::min<int64_t>(S2_GROUP, nf - base);
        double R[S2_GROUP + 1];
        R[n] = 1.0;
        for (int64_t i = n - 1; i >= 0; i--) R[i] = R[i + 1] * (1.0 - P->h_fault_p[base + i]);
        G[g] = threshold_q(1.0 - R[0]);
        int64_t last = -1;
        for (int64_t i = 0; i < n; i++)
            if (P->h_fault_p[base + i] > 0.0) last = i;
        for (int64_t i = 0; i < n; i++) {
            const double pi = P->h_fault_p[base + i];
            const int64_t c = fault[base + i];
            const uint32_t Q = i == last ? 4294967295u : threshold_q(pi / (1.0 - R[i]));
            const uint32_t k = kind[c] == CK_DEP1 ? CK_DEP1 : kind[c] == CK_DEP2 ? CK_DEP2 : CK_BERN;
            ch[base + i] = make_uint4(Q, threshold_q(pi), sym0[c] - 1u, k | (i == last ? S2_LAST : 0u));
        }
    }
    for (size_t q = 0; q < G4.size(); q++) G4[q] = make_uint4(G[4 * q], G[4 * q + 1], G[4 * q + 2], G[4 * q + 3]);
    sp_status st;
    if ((st = upload_vec(&P->d_s2Ch, ch, s)) || (st = upload_vec(&P->d_s2G, G4, s)) || (st = upload_vec(&P->d_s2Rand, rnd, s))) {
        dev_free(P->d_s2Ch);
        dev_free(P->d_s2G);
        dev_free(P->d_s2Rand);
        P->d_s2Ch = nullptr;
        P->d_s2G = nullptr;
        P->d_s2Rand = nullptr;
        return st;
    }
    SP_CUDA(cudaStreamSynchronize(s));
    P->s2_nfault = nf;
    P->s2_ngrp = ngrp;
    P->s2_nrnd = (int64_t)rnd.size();
    return SP_OK;
}

sp_status grouped_chunk(sp_program *P, uint64_t seed, uint64_t shot0, uint64_t nshots, uint64_t *d_meas,
                        uint64_t *d_det, uint64_t *d_obs, cudaStream_t s)
{
    if (nshots == 0) return SP_OK;
    if (!P->fused_tw || !P->d_s2Ch) return set_error(SP_ERR_INVALID_ARG, "the grouped draw needs the fused path");
    const FusedParams fp = fused_params(P, P->fused_tw, seed, shot0, nshots, d_meas, d_det, d_obs);
    GroupedFn fn = grouped_kernel(P->fused_tw, P->fused_unroll);
    const int cfg = 16 * P->fused_tw + P->fused_unroll;
    if (P->s2_cfg != cfg) {
        SP_CUDA(max_dynamic_smem(fn));
        int occ = 0;
        SP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, P->fused_threads, P->fused_smem));
        P->s2_ctas_per_sm = std::max(occ, 1);
        P->s2_cfg = cfg;
    }
    const int occ = P->s2_ctas_per_sm;
    const uint64_t per_tile = 32u * (uint64_t)P->fused_tw;
    const uint64_t ntiles = (nshots + per_tile - 1) / per_tile;
    const uint64_t grid = std::min<uint64_t>(ntiles, (uint64_t)P->num_sms * (uint64_t)std::max(occ, 1));
    ProfScope ps(P, SP_KERNEL_FUSED, s);
    fn<<<dim3((unsigned)grid), dim3((unsigned)P->fused_threads), P->fused_smem, s>>>(fp);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

}  // namespace sp
