// sp_fused.cu -- the sampling hot path fused into one persistent kernel.
//
// Algorithm 1 "Sampling" (arXiv 2311.03906, Sec. 3.2.3, Eq. sampling) for a
// tile of 32*TW shots per CTA iteration, entirely in shared memory:
//   phase 1  draw: Philox4x32-10 keyed by (seed, shot, channel/4); each warp
//            owns a contiguous range of 4-channel blocks, lane = shot, and
//            writes the bit-sliced fault word of every symbol of its range
//            (bit = shot within the tile) into the tile B_s;
//   phase 2  product: (A) every measurement row's own part, c'_j ^ XOR of
//            B_s over its delta symbols, for all rows in parallel; (B) the
//            parent chains m_j ^= m_parent; (C) detectors and observables as
//            XORs of their measurement records, which is their definition;
//   phase 3  emit: 32x32 warp transposes turn the bit-sliced rows into
//            shot-major packed words, staged in shared memory and written as
//            contiguous per-shot segments.
// Nothing but the records touches HBM.  The same draw code also serves the
// staged path (fault bits to global memory) used when the tile does not fit.
//
// Philox per (shot, channel block b): counter (shot lo, shot hi, b, 0).
// Round 1's product M1*b is the same for every lane (one per warp), and the
// products M0*(shot lo) of round 1 and M1*(hi0 ^ k1) of round 2 do not depend
// on b, so they are computed once per shot: 17 of the 20 wide multiplies of a
// block remain per (shot, block).
#include <algorithm>
#include <numeric>
#include <vector>

#include "sp_internal.h"

namespace sp {

constexpr uint32_t FM = 0xffffffffu;
constexpr uint32_t PH_M0 = 0xD2511F53u, PH_M1 = 0xCD9E8D57u;
constexpr uint32_t PH_W0 = 0x9E3779B9u, PH_W1 = 0xBB67AE85u;
constexpr int FUSED_THREADS = 512;

__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane)
{
    const uint32_t m16 = 0x0000FFFFu, m8 = 0x00FF00FFu, m4 = 0x0F0F0F0Fu, m2 = 0x33333333u, m1 = 0x55555555u;
    uint32_t y;
    y = __shfl_xor_sync(FM, x, 16); x = (lane & 16) ? ((x & ~m16) | ((y >> 16) & m16)) : ((x & m16) | ((y & m16) << 16));
    y = __shfl_xor_sync(FM, x, 8);  x = (lane & 8) ? ((x & ~m8) | ((y >> 8) & m8)) : ((x & m8) | ((y & m8) << 8));
    y = __shfl_xor_sync(FM, x, 4);  x = (lane & 4) ? ((x & ~m4) | ((y >> 4) & m4)) : ((x & m4) | ((y & m4) << 4));
    y = __shfl_xor_sync(FM, x, 2);  x = (lane & 2) ? ((x & ~m2) | ((y >> 2) & m2)) : ((x & m2) | ((y & m2) << 2));
    y = __shfl_xor_sync(FM, x, 1);  x = (lane & 1) ? ((x & ~m1) | ((y >> 1) & m1)) : ((x & m1) | ((y & m1) << 1));
    return x;
}

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

// Rounds 1..10 of Philox4x32-10 for counter (shot, b): uhi/ulo = M1*b.
__device__ __forceinline__ void philox_block(const ShotConst &s, uint32_t uhi, uint32_t ulo, uint32_t k0,
                                             uint32_t k1, uint32_t &o0, uint32_t &o1, uint32_t &o2, uint32_t &o3)
{
    // round 1 (counter word 3 is 0)
    uint32_t x0 = uhi ^ s.c1 ^ k0;
    // round 2
    const uint64_t p = (uint64_t)PH_M0 * x0;
    uint32_t c0 = s.r2hi ^ ulo ^ (k0 + PH_W0);
    uint32_t c1 = s.r2lo;
    uint32_t c2 = (uint32_t)(p >> 32) ^ s.x3 ^ (k1 + PH_W1);
    uint32_t c3 = (uint32_t)p;
#pragma unroll
    for (int r = 2; r < 10; r++) {
        const uint64_t p0 = (uint64_t)PH_M0 * c0;
        const uint64_t p1 = (uint64_t)PH_M1 * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ (k0 + (uint32_t)r * PH_W0);
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ (k1 + (uint32_t)r * PH_W1);
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
    }
    o0 = c0; o1 = c1; o2 = c2; o3 = c3;
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

// Draw the symbols of blocks [b0, b1) for TW shots per lane (shot words
// w_t = 32-shot groups).  Each flushed 32-symbol column group is handed to
// sink(symbol base, lane's column words[TW]) with the lane's symbol = base+lane.
template <int TW> struct Cols { uint32_t v[TW]; };
template <int TW> struct Shots { ShotConst s[TW]; };

template <int TW, typename Sink>
__device__ __forceinline__ void draw_blocks(const uint4 *__restrict__ blkT, const uint32_t *__restrict__ blkMeta,
                                            int64_t b0, int64_t b1, uint32_t sym_begin, const Shots<TW> sc,
                                            uint32_t k0, uint32_t k1, int lane, Sink sink)
{
    uint64_t acc[TW];
#pragma unroll
    for (int t = 0; t < TW; t++) acc[t] = 0;
    uint32_t fill = 0, base = sym_begin;
    for (int64_t b = b0; b < b1; b++) {
        const uint4 T = blkT[b];
        const uint32_t meta = blkMeta[b];
        const uint64_t u = (uint64_t)PH_M1 * (uint32_t)b;
        const uint32_t uhi = (uint32_t)(u >> 32), ulo = (uint32_t)u;
        uint32_t r[TW][4];
        bool fire = false;
#pragma unroll
        for (int t = 0; t < TW; t++) {
            philox_block(sc.s[t], uhi, ulo, k0, k1, r[t][0], r[t][1], r[t][2], r[t][3]);
            fire |= (r[t][0] < T.x) | (r[t][1] < T.y) | (r[t][2] < T.z) | (r[t][3] < T.w);
        }
        if (__any_sync(FM, fire)) {
            const uint32_t Ts[4] = {T.x, T.y, T.z, T.w};
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const uint32_t kind = (meta >> (2 * i)) & 3u;
                const uint32_t off = fill + ((meta >> (8 + 4 * i)) & 15u);
#pragma unroll
                for (int t = 0; t < TW; t++) acc[t] |= (uint64_t)chan_bits(r[t][i], Ts[i], kind) << off;
            }
        }
        fill += meta >> 24;
        if (fill >= 32) {
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
        }
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

struct FusedParams {
    const uint4 *blkT;
    const uint32_t *blkMeta;
    const uint32_t *blkSym0;
    int64_t n_blk;
    int64_t n_sym, n_rows, n_meas, n_det, n_obs;
    const uint4 *aItem;        // step A: {index-group offset, group count, row, const flag}
    const uint32_t *aOff;      // [threads + 1]
    const uint2 *bItem;        // step B: (row, parent), parents first within a thread
    const uint32_t *bOff;      // [threads + 1]
    const uint32_t *cOff;      // step C: detector/observable t = XOR of measurement rows
    const uint32_t *cRefs;
    const uint4 *idx4;         // groups of 4 (u32) or 8 (u16) symbol indices
    uint64_t seed, shot0, nshots;
    uint64_t *out[3];
    int64_t rows0[3], nrow[3];
    uint32_t rec_off_words;   // offset of R_s in shared memory (u32 words)
};

template <int TW> struct TileWord;
template <> struct TileWord<1> {
    typedef uint32_t T;
    __device__ static T zero() { return 0u; }
    __device__ static T ones() { return FM; }
    __device__ static uint32_t get(T v, int) { return v; }
    __device__ static T make(const Cols<1> c) { return c.v[0]; }
};
template <> struct TileWord<2> {
    typedef uint2 T;
    __device__ static T zero() { return make_uint2(0u, 0u); }
    __device__ static T ones() { return make_uint2(FM, FM); }
    __device__ static uint32_t get(T v, int t) { return t ? v.y : v.x; }
    __device__ static T make(const Cols<2> c) { return make_uint2(c.v[0], c.v[1]); }
};
__device__ __forceinline__ uint32_t xorw(uint32_t a, uint32_t b) { return a ^ b; }
__device__ __forceinline__ uint2 xorw(uint2 a, uint2 b) { return make_uint2(a.x ^ b.x, a.y ^ b.y); }

template <typename W>
__device__ __forceinline__ W gather4(const W *Bs, uint4 s)
{
    return xorw(xorw(Bs[s.x], Bs[s.y]), xorw(Bs[s.z], Bs[s.w]));
}

template <typename W>
__device__ __forceinline__ W gather8(const W *Bs, uint4 s)
{
    const W a = xorw(xorw(Bs[s.x & 0xffffu], Bs[s.x >> 16]), xorw(Bs[s.y & 0xffffu], Bs[s.y >> 16]));
    const W b = xorw(xorw(Bs[s.z & 0xffffu], Bs[s.z >> 16]), xorw(Bs[s.w & 0xffffu], Bs[s.w >> 16]));
    return xorw(a, b);
}

template <int TW, bool IDX16>
__global__ void __launch_bounds__(FUSED_THREADS, (TW == 1 ? 2 : 1)) k_fused(FusedParams p)
{
    typedef TileWord<TW> TWd;
    typedef typename TWd::T W;
    extern __shared__ __align__(16) uint32_t sm[];
    W *Bs = reinterpret_cast<W *>(sm);                       // n_sym + 1 (last = zero)
    W *Rs = reinterpret_cast<W *>(sm + p.rec_off_words);     // n_rows
    uint32_t *stage = sm;                                    // aliases Bs in phase 3
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const uint64_t per_tile = 32u * TW;
    const uint64_t ntiles = (p.nshots + per_tile - 1) / per_tile;
    const int64_t b0 = (int64_t)warp * p.n_blk / nwarps, b1 = (int64_t)(warp + 1) * p.n_blk / nwarps;
    const uint32_t sbeg = p.blkSym0[b0], send = p.blkSym0[b1];
    const uint32_t k0 = (uint32_t)p.seed, k1 = (uint32_t)(p.seed >> 32);

    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t trel = tile * per_tile;
        // ---- phase 1: draw ------------------------------------------------
        Shots<TW> sc;
#pragma unroll
        for (int t = 0; t < TW; t++) sc.s[t] = shot_const(p.shot0 + trel + 32u * t + lane, k1);
        if (tid == 0) Bs[p.n_sym] = TWd::zero();
        draw_blocks<TW>(p.blkT, p.blkMeta, b0, b1, sbeg, sc, k0, k1, lane,
                        [=](uint32_t base, const Cols<TW> col) {
                            if (base + lane < send) Bs[base + lane] = TWd::make(col);
                        });
        __syncthreads();
        // ---- phase 2: GF(2) product ------------------------------------------
        // A: every measurement row's own part c'_j ^ XOR of B_s over its delta
        //    symbols; rows are independent, balanced over threads.
        {
            const uint32_t e = p.aOff[tid + 1];
            for (uint32_t i = p.aOff[tid]; i < e; i++) {
                const uint4 m = p.aItem[i];
                W acc = m.w ? TWd::ones() : TWd::zero();
                const uint4 *q = p.idx4 + m.x;
                uint32_t k = 0;
                if (IDX16) {
                    for (; k + 2 <= m.y; k += 2) {
                        const uint4 s0 = q[k], s1 = q[k + 1];
                        acc = xorw(acc, xorw(gather8(Bs, s0), gather8(Bs, s1)));
                    }
                    if (k < m.y) acc = xorw(acc, gather8(Bs, q[k]));
                } else {
                    for (; k + 4 <= m.y; k += 4) {
                        const uint4 s0 = q[k], s1 = q[k + 1], s2 = q[k + 2], s3 = q[k + 3];
                        acc = xorw(acc, xorw(gather4(Bs, s0), gather4(Bs, s1)));
                        acc = xorw(acc, xorw(gather4(Bs, s2), gather4(Bs, s3)));
                    }
                    for (; k < m.y; k++) acc = xorw(acc, gather4(Bs, q[k]));
                }
                Rs[m.z] = acc;
            }
        }
        __syncthreads();
        // B: parent chains, m_j = own part ^ m_parent (each thread owns whole
        //    trees and walks them parents first).
        {
            const uint32_t e = p.bOff[tid + 1];
            for (uint32_t i = p.bOff[tid]; i < e; i++) {
                const uint2 rp = p.bItem[i];
                Rs[rp.x] = xorw(Rs[rp.x], Rs[rp.y]);
            }
        }
        __syncthreads();
        // C: detectors and observables are XORs of measurement records.
        for (int64_t t = tid; t < p.n_det + p.n_obs; t += blockDim.x) {
            W acc = TWd::zero();
            for (uint32_t k = p.cOff[t]; k < p.cOff[t + 1]; k++) acc = xorw(acc, Rs[p.cRefs[k]]);
            Rs[p.n_meas + t] = acc;
        }
        __syncthreads();
        // ---- phase 3: emit shot-major records ------------------------------
#pragma unroll
        for (int sg = 0; sg < 3; sg++) {
            uint64_t *dst = p.out[sg];
            const int64_t n = p.nrow[sg];
            if (!dst || n == 0) continue;
            const int64_t row0 = p.rows0[sg];
            const int words32 = (int)(2 * ((n + 63) / 64));
            const int stride = words32 + 1;
            for (int g = warp; g < words32; g += nwarps) {
                const int64_t r = 32 * (int64_t)g + lane;
#pragma unroll
                for (int t = 0; t < TW; t++) {
                    const uint32_t x = r < n ? TWd::get(Rs[row0 + r], t) : 0u;
                    stage[(32 * t + lane) * stride + g] = __any_sync(FM, x != 0u) ? transpose32(x, lane) : 0u;
                }
            }
            __syncthreads();
            uint32_t *o32 = reinterpret_cast<uint32_t *>(dst);
            for (int sh = warp; sh < 32 * TW; sh += nwarps) {
                const uint64_t shot = trel + (uint64_t)sh;
                if (shot >= p.nshots) continue;
                uint32_t *o = o32 + shot * (uint64_t)words32;
                for (int g = lane; g < words32; g += 32) o[g] = stage[sh * stride + g];
            }
            __syncthreads();
        }
    }
}

// Staged draw: fault bits to global memory, bit-sliced [symbol][32-shot word].
// Block = 8 warps; warp = one 32-shot word over all channel blocks.
__global__ void __launch_bounds__(256) k_draw_staged(const uint4 *__restrict__ blkT,
                                                     const uint32_t *__restrict__ blkMeta, int64_t n_blk,
                                                     int64_t n_sym, uint64_t seed, uint64_t shot0, int64_t nwords,
                                                     uint32_t *__restrict__ B, int64_t bpitch)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (w >= nwords) return;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    Shots<1> sc;
    sc.s[0] = shot_const(shot0 + (uint64_t)w * 32u + (uint64_t)lane, k1);
    draw_blocks<1>(blkT, blkMeta, 0, n_blk, 0u, sc, k0, k1, lane,
                   [=](uint32_t base, const Cols<1> col) {
                       if ((int64_t)base + lane < n_sym) B[(size_t)(base + lane) * bpitch + w] = col.v[0];
                   });
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {
template <typename T>
sp_status upload(T **dst, const std::vector<T> &src, cudaStream_t s)
{
    const size_t n = std::max<size_t>(src.size(), 1);
    if (cudaMalloc((void **)dst, n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *dst = nullptr;
        return set_error(SP_ERR_OOM, "cudaMalloc of the sampler program failed");
    }
    if (!src.empty()) SP_CUDA(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return SP_OK;
}
}  // namespace

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
    std::vector<uint32_t> bMeta((size_t)nb), bSym0((size_t)nb + 1, 0);
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
    if ((st = upload(&P->d_blkT, bT, s)) || (st = upload(&P->d_blkMeta, bMeta, s)) || (st = upload(&P->d_blkSym0, bSym0, s)))
        return st;

    // ---- level-ordered, padded product program ----------------------------
    const int64_t R = P->n_rows;
    std::vector<int32_t> parent((size_t)R);
    std::vector<uint8_t> cflag((size_t)R);
    std::vector<uint32_t> off((size_t)R + 1);
    std::vector<uint32_t> idx((size_t)P->nnz_delta);
    if (R) {
        SP_CUDA(cudaMemcpyAsync(parent.data(), P->d_parent, (size_t)R * 4, cudaMemcpyDeviceToHost, s));
        SP_CUDA(cudaMemcpyAsync(cflag.data(), P->d_cflag, (size_t)R, cudaMemcpyDeviceToHost, s));
        SP_CUDA(cudaMemcpyAsync(off.data(), P->d_rowOff, ((size_t)R + 1) * 4, cudaMemcpyDeviceToHost, s));
        if (!idx.empty())
            SP_CUDA(cudaMemcpyAsync(idx.data(), P->d_idx, idx.size() * 4, cudaMemcpyDeviceToHost, s));
        SP_CUDA(cudaStreamSynchronize(s));
    }
    // Step A: the own part of every measurement row (its delta symbols and
    // constant) -- independent rows, longest first to the least loaded thread.
    // Step B: parent chains -- whole trees per thread, parents first.
    // Step C: detectors and observables from their measurement records.
    const int64_t M = P->n_meas;
    const bool idx16 = P->n_sym < 65535;
    const uint32_t per_group = idx16 ? 8u : 4u;
    const int NT = FUSED_THREADS;
    auto lpt = [&](const std::vector<int64_t> &items, const std::vector<double> &cost, std::vector<int32_t> &owner_of) {
        std::vector<std::pair<double, int>> heap;
        for (int t = 0; t < NT; t++) heap.push_back({0.0, t});
        auto cmp = [](const std::pair<double, int> &a, const std::pair<double, int> &b) {
            return a.first > b.first || (a.first == b.first && a.second > b.second);
        };
        std::make_heap(heap.begin(), heap.end(), cmp);
        double mx = 0.0;
        for (int64_t it : items) {
            std::pop_heap(heap.begin(), heap.end(), cmp);
            auto hh = heap.back();
            heap.pop_back();
            owner_of[it] = hh.second;
            hh.first += cost[it];
            mx = std::max(mx, hh.first);
            heap.push_back(hh);
            std::push_heap(heap.begin(), heap.end(), cmp);
        }
        return mx;
    };
    std::vector<uint32_t> groups((size_t)M);
    std::vector<double> costA((size_t)M);
    std::vector<int64_t> itemsA((size_t)M);
    for (int64_t j = 0; j < M; j++) {
        groups[j] = (off[j + 1] - off[j] + per_group - 1) / per_group;
        costA[j] = 1.0 + groups[j];
        itemsA[j] = j;
    }
    std::stable_sort(itemsA.begin(), itemsA.end(), [&](int64_t a, int64_t b) { return costA[a] > costA[b]; });
    std::vector<int32_t> ownerA((size_t)M, 0);
    P->fused_max_load = lpt(itemsA, costA, ownerA);
    // index groups laid out per measurement row
    std::vector<uint4> idx4;
    std::vector<uint32_t> goff((size_t)M);
    const uint32_t zero = (uint32_t)P->n_sym;   // index of the zero slot
    for (int64_t j = 0; j < M; j++) {
        const uint32_t a = off[j], e = off[j + 1];
        goff[j] = (uint32_t)idx4.size();
        for (uint32_t k = 0; k < groups[j]; k++) {
            uint32_t v[8];
            for (uint32_t i = 0; i < per_group; i++) {
                const uint32_t at = a + per_group * k + i;
                v[i] = at < e ? idx[at] : zero;
            }
            if (idx16)
                idx4.push_back(make_uint4(v[0] | (v[1] << 16), v[2] | (v[3] << 16), v[4] | (v[5] << 16), v[6] | (v[7] << 16)));
            else
                idx4.push_back(make_uint4(v[0], v[1], v[2], v[3]));
        }
    }
    std::vector<uint32_t> aOff((size_t)NT + 1, 0);
    for (int64_t j = 0; j < M; j++) aOff[ownerA[j] + 1]++;
    for (int t = 0; t < NT; t++) aOff[t + 1] += aOff[t];
    std::vector<uint4> aItem((size_t)M);
    {
        std::vector<uint32_t> pos(aOff.begin(), aOff.end() - 1);
        for (int64_t j : itemsA)
            aItem[pos[ownerA[j]]++] = make_uint4(goff[j], groups[j], (uint32_t)j, (uint32_t)cflag[j]);
    }
    // step B: trees of measurement rows (parents of measurement rows are
    // earlier measurement rows)
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
    lpt(trees, tsize, ownerT);
    std::vector<uint32_t> bOff((size_t)NT + 1, 0);
    for (int64_t j = 0; j < M; j++) if (parent[j] >= 0) bOff[ownerT[root[j]] + 1]++;
    for (int t = 0; t < NT; t++) bOff[t + 1] += bOff[t];
    std::vector<uint2> bItem((size_t)bOff[NT]);
    {
        std::vector<uint32_t> pos(bOff.begin(), bOff.end() - 1);
        for (int64_t j = 0; j < M; j++)   // increasing j: parents before children
            if (parent[j] >= 0) bItem[pos[ownerT[root[j]]]++] = make_uint2((uint32_t)j, (uint32_t)parent[j]);
    }
    P->fused_idx16 = idx16;
    if ((st = upload(&P->d_fRowMeta, aItem, s)) || (st = upload(&P->d_fAOff, aOff, s)) ||
        (st = upload(&P->d_fChain, bItem, s)) || (st = upload(&P->d_fBOff, bOff, s)) ||
        (st = upload(&P->d_fCOff, P->h_xoff, s)) || (st = upload(&P->d_fCRefs, P->h_xrefs, s)) ||
        (st = upload(&P->d_fIdx4, idx4, s)))
        return st;
    P->fused_idx4 = (int64_t)idx4.size();
    // the fused program needs measurement rows to have measurement parents
    for (int64_t j = 0; j < M; j++)
        if (parent[j] >= M) return set_error(SP_ERR_CUDA, "measurement row with a non-measurement parent");

    // ---- shared-memory footprint and occupancy of the fused kernel --------
    int dev = 0, smem_max = 0, nsm = 0;
    SP_CUDA(cudaGetDevice(&dev));
    SP_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    SP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    P->num_sms = nsm;
    P->fused_tw = 0;
    int64_t max_words32 = 0;
    for (int64_t n : {P->n_meas, P->n_det, P->n_obs}) max_words32 = std::max<int64_t>(max_words32, 2 * ((n + 63) / 64));
    for (int tw : {2, 1}) {
        const int64_t bwords = ((P->n_sym + 1) * tw + 3) / 4 * 4;
        const int64_t rwords = R * tw;
        const int64_t stage_words = 32 * tw * (max_words32 + 1);
        const int64_t words = std::max(bwords, stage_words) + rwords;
        const int64_t bytes = words * 4;
        if (bytes <= smem_max && R > 0 && nb > 0) {
            P->fused_tw = tw;
            P->fused_smem = (size_t)bytes;
            P->fused_rec_off = (uint32_t)std::max(bwords, stage_words);
            break;
        }
    }
    if (P->fused_tw) {
        void (*fn)(FusedParams) = P->fused_tw == 2 ? (P->fused_idx16 ? k_fused<2, true> : k_fused<2, false>)
                                                   : (P->fused_idx16 ? k_fused<1, true> : k_fused<1, false>);
        SP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P->fused_smem));
        int occ = 0;
        SP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, FUSED_THREADS, P->fused_smem));
        P->fused_ctas_per_sm = std::max(occ, 1);
    }
    return SP_OK;
}

sp_status launch_draw_staged(const sp_program *P, uint64_t seed, uint64_t shot0, int64_t nwords, uint32_t *B,
                             int64_t pitch, cudaStream_t s)
{
    if (P->n_sym == 0 || nwords == 0) return SP_OK;
    k_draw_staged<<<(unsigned)ceil_div(nwords, 8), 256, 0, s>>>(P->d_blkT, P->d_blkMeta, P->n_blk, P->n_sym, seed,
                                                                 shot0, nwords, B, pitch);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

sp_status fused_chunk(sp_program *P, uint64_t seed, uint64_t shot0, uint64_t nshots, uint64_t *d_meas,
                      uint64_t *d_det, uint64_t *d_obs, cudaStream_t s)
{
    if (nshots == 0) return SP_OK;
    if (!P->fused_tw) return set_error(SP_ERR_INVALID_ARG, "fused path unavailable for this program");
    FusedParams fp;
    fp.blkT = P->d_blkT; fp.blkMeta = P->d_blkMeta; fp.blkSym0 = P->d_blkSym0; fp.n_blk = P->n_blk;
    fp.n_sym = P->n_sym; fp.n_rows = P->n_rows; fp.n_meas = P->n_meas; fp.n_det = P->n_det; fp.n_obs = P->n_obs;
    fp.aItem = P->d_fRowMeta; fp.aOff = P->d_fAOff; fp.bItem = P->d_fChain; fp.bOff = P->d_fBOff;
    fp.cOff = P->d_fCOff; fp.cRefs = P->d_fCRefs; fp.idx4 = P->d_fIdx4;
    fp.seed = seed; fp.shot0 = shot0; fp.nshots = nshots;
    fp.out[0] = d_meas; fp.out[1] = d_det; fp.out[2] = d_obs;
    fp.rows0[0] = 0; fp.rows0[1] = P->n_meas; fp.rows0[2] = P->n_meas + P->n_det;
    fp.nrow[0] = P->n_meas; fp.nrow[1] = P->n_det; fp.nrow[2] = P->n_obs;
    fp.rec_off_words = P->fused_rec_off;
    const uint64_t per_tile = 32u * (uint64_t)P->fused_tw;
    const uint64_t ntiles = (nshots + per_tile - 1) / per_tile;
    const uint64_t grid = std::min<uint64_t>(ntiles, (uint64_t)P->num_sms * (uint64_t)P->fused_ctas_per_sm);
    ProfScope ps(P, SP_KERNEL_FUSED, s);
    const dim3 g((unsigned)grid), b(FUSED_THREADS);
    if (P->fused_tw == 2) {
        if (P->fused_idx16) k_fused<2, true><<<g, b, P->fused_smem, s>>>(fp);
        else k_fused<2, false><<<g, b, P->fused_smem, s>>>(fp);
    } else {
        if (P->fused_idx16) k_fused<1, true><<<g, b, P->fused_smem, s>>>(fp);
        else k_fused<1, false><<<g, b, P->fused_smem, s>>>(fp);
    }
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

}  // namespace sp
