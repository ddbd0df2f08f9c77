// sp_sample.cu -- Algorithm 1 "Sampling" on the GPU (arXiv 2311.03906,
// Sec. 3.2.3, Eq. sampling): draw b for every shot from the noise model,
// then M = [m_1; ...; m_nm] . [b_1 ... b_nsmp] over GF(2).
//
//   K4 k_draw_staged (sp_fused.cu)  Philox4x32-10 per (seed, shot,
//                 channel/4); lane = shot; the channel's symbol bits (Sec. 3.1
//                 distributions) are packed 32 symbols at a time and
//                 transposed across the warp into bit-sliced words
//                 B[s-1][shot/32] (bit = shot % 32).
//   K5 k_gather   the GF(2) product in sparse form: record row j of a
//                 32-shot word is c'_j ^ rec[parent(j)] ^ XOR_{s in delta_j}
//                 B[s-1], lane = 32-shot word, so every index load is shared
//                 by 1024 shots and every B load is a coalesced 128-byte row
//                 segment; with few shots, k_gather_full takes each row
//                 from its full symbol list instead, all rows at once.
//   K6 k_emit     32x32 bit transposes from the bit-sliced records to the
//                 shot-major packed output.
#include <algorithm>
#include <vector>

#include "sp_internal.h"

namespace sp {

constexpr uint32_t FULLM = 0xffffffffu;
// Largest record block the push path keeps (it must stay in L2 for the atomics).
constexpr uint64_t PUSH_MAX_BYTES = 96ull << 20;
// The push draw's queued events address a warp's channel blocks in 25 bits.
constexpr int64_t PUSH_MAX_BLOCKS = (int64_t)1 << 25;


// K5.  Warp = 1024 shots (lane = 32-shot word); rows in order so a parent
// is always finished (by the same lane) before its children.
__global__ void __launch_bounds__(128) k_gather(const uint32_t *__restrict__ B, int64_t bpitch,
                                                int64_t nwords, const uint32_t *__restrict__ rowOff,
                                                const uint32_t *__restrict__ idx,
                                                const int32_t *__restrict__ parent,
                                                const uint8_t *__restrict__ cflag, int64_t nrows,
                                                uint32_t *recT, int64_t rpitch)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32 + lane;
    if (((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32 >= nwords) return;
    const bool ok = w < nwords;
    const uint32_t *Bw = B + w;
    for (int64_t j = 0; j < nrows; j++) {
        uint32_t acc = cflag[j] ? FULLM : 0u;
        const int32_t p = parent[j];
        if (p >= 0 && ok) acc ^= recT[(size_t)p * rpitch + w];
        const uint32_t e = rowOff[j + 1];
        uint32_t k = rowOff[j];
        uint32_t a1 = 0, a2 = 0, a3 = 0;
        if (ok) {
            for (; k + 4 <= e; k += 4) {
                const uint32_t s0 = idx[k], s1 = idx[k + 1], s2 = idx[k + 2], s3 = idx[k + 3];
                acc ^= Bw[(size_t)s0 * bpitch];
                a1 ^= Bw[(size_t)s1 * bpitch];
                a2 ^= Bw[(size_t)s2 * bpitch];
                a3 ^= Bw[(size_t)s3 * bpitch];
            }
            for (; k < e; k++) acc ^= Bw[(size_t)idx[k] * bpitch];
            recT[(size_t)j * rpitch + w] = acc ^ a1 ^ a2 ^ a3;
        }
    }
}

// K5 for few shots.  Warp = (record row j, 32 consecutive 32-shot words),
// lane = word: row j from its full symbol list (not its delta against a
// parent), so that rows are independent and all of them run at once.
__global__ void __launch_bounds__(256) k_gather_full(const uint32_t *__restrict__ B, int64_t bpitch,
                                                     int64_t nwords, const uint32_t *__restrict__ fullOff,
                                                     const uint32_t *__restrict__ fullIdx,
                                                     const uint8_t *__restrict__ cst, int64_t nrows,
                                                     uint32_t *recT, int64_t rpitch)
{
    const int lane = threadIdx.x & 31;
    const int64_t wgroups = (nwords + 31) / 32;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t j = gw / wgroups;
    if (j >= nrows) return;
    const int64_t w = (gw % wgroups) * 32 + lane;
    if (w >= nwords) return;
    const uint32_t *Bw = B + w;
    uint32_t acc = cst[j] ? FULLM : 0u, a1 = 0, a2 = 0, a3 = 0;
    const uint32_t e = fullOff[j + 1];
    uint32_t k = fullOff[j];
    for (; k + 4 <= e; k += 4) {
        acc ^= Bw[(size_t)fullIdx[k] * bpitch];
        a1 ^= Bw[(size_t)fullIdx[k + 1] * bpitch];
        a2 ^= Bw[(size_t)fullIdx[k + 2] * bpitch];
        a3 ^= Bw[(size_t)fullIdx[k + 3] * bpitch];
    }
    for (; k < e; k++) acc ^= Bw[(size_t)fullIdx[k] * bpitch];
    recT[(size_t)j * rpitch + w] = acc ^ a1 ^ a2 ^ a3;
}

// K6.  Block = 256 threads; tile = 256 record rows x 8 words (256 shots).
// Word w of row j is recT[j * rstride + w * wstride] (row-major records:
// rstride = pitch, wstride = 1; word-major: rstride = 1, wstride = rows).
// Transposes 32x32 blocks with warp shuffles and writes 32 contiguous bytes
// per shot.
__global__ void __launch_bounds__(256) k_emit(const uint32_t *__restrict__ recT, int64_t rstride, int64_t wstride,
                                              int64_t row0, int64_t nrows, int64_t nshots,
                                              uint32_t *__restrict__ out, int64_t out_words32)
{
    __shared__ uint32_t in_t[256][9];
    __shared__ uint32_t out_t[256][9];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t rb = (int64_t)blockIdx.y * 256;   // first row (segment-relative)
    const int64_t wb = (int64_t)blockIdx.x * 8;     // first 32-shot word
    const int64_t nwords = (nshots + 31) / 32;
    {
        const int64_t r = rb + t;
        for (int k = 0; k < 8; k++) {
            uint32_t v = 0;
            if (r < nrows && wb + k < nwords) v = recT[(size_t)(row0 + r) * rstride + (size_t)(wb + k) * wstride];
            in_t[t][k] = v;
        }
    }
    __syncthreads();
    // 64 (row group, word) blocks, 8 per warp
    for (int q = warp; q < 64; q += 8) {
        const int g = q >> 3, k = q & 7;
        const uint32_t x = in_t[g * 32 + lane][k];
        out_t[k * 32 + lane][g] = transpose32(x, lane);
    }
    __syncthreads();
    const int64_t shot = wb * 32 + t;
    if (shot < nshots) {
        const int64_t word0 = rb / 32;   // first u32 word of this row chunk
        uint32_t *dst = out + (size_t)shot * out_words32 + word0;
        for (int g = 0; g < 8; g++)
            if (word0 + g < out_words32) dst[g] = out_t[t][g];
    }
}

// Symbol -> rows index of the full rows (counting sort by symbol; the order
// of the rows within one symbol's list is not fixed, and XOR does not need
// it): pass 1 counts, pass 2 places each (row, symbol) at its symbol's next
// free slot.  One warp per row.
__global__ void k_col_count(const uint32_t *__restrict__ off, const uint32_t *__restrict__ idx, int64_t nrows,
                            uint32_t *cnt)
{
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (j >= nrows) return;
    for (uint32_t k = off[j] + (threadIdx.x & 31); k < off[j + 1]; k += 32) atomicAdd(&cnt[idx[k]], 1u);
}

__global__ void k_col_fill(const uint32_t *__restrict__ off, const uint32_t *__restrict__ idx, int64_t nrows,
                           uint32_t *next, uint32_t *rows)
{
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (j >= nrows) return;
    for (uint32_t k = off[j] + (threadIdx.x & 31); k < off[j + 1]; k += 32) rows[atomicAdd(&next[idx[k]], 1u)] = (uint32_t)j;
}

// The rows of each symbol (transpose of the kept full rows), built on the
// first sample that pushes fired symbols into the records; it synchronises
// the stream once.  On an error nothing is kept and the program stays usable.
static sp_status ensure_colfull(sp_program *P, cudaStream_t s)
{
    if (P->d_colFullRows) return SP_OK;
    uint32_t *cnt = nullptr, *off = nullptr, *rows = nullptr;
    auto fail = [&](sp_status st, const char *what) {
        cudaGetLastError();
        dev_free(cnt);
        dev_free(off);
        dev_free(rows);
        return set_error(st, what);
    };
    if (dev_alloc((void **)&cnt, (size_t)P->n_sym * 4) != cudaSuccess)
        return fail(SP_ERR_OOM, "cudaMalloc of the symbol -> rows index failed");
    if (cudaMemsetAsync(cnt, 0, (size_t)P->n_sym * 4, s) != cudaSuccess)
        return fail(SP_ERR_CUDA, "building the symbol -> rows index failed");
    const unsigned rb = (unsigned)ceil_div(P->n_rows, 8);
    k_col_count<<<rb, 256, 0, s>>>(P->d_fullOff, P->d_fullIdx, P->n_rows, cnt);
    std::vector<uint32_t> c((size_t)P->n_sym), o((size_t)P->n_sym + 1, 0);
    if (cudaMemcpyAsync(c.data(), cnt, (size_t)P->n_sym * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(SP_ERR_CUDA, "building the symbol -> rows index failed");
    uint64_t acc = 0;
    for (int64_t q = 0; q < P->n_sym; q++) { o[q] = (uint32_t)acc; acc += c[q]; }
    o[P->n_sym] = (uint32_t)acc;
    if (dev_alloc((void **)&off, ((size_t)P->n_sym + 1) * 4) != cudaSuccess ||
        dev_alloc((void **)&rows, (size_t)std::max<uint64_t>(acc, 1) * 4) != cudaSuccess)
        return fail(SP_ERR_OOM, "cudaMalloc of the symbol -> rows index failed");
    if (cudaMemcpyAsync(off, o.data(), ((size_t)P->n_sym + 1) * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(cnt, o.data(), (size_t)P->n_sym * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return fail(SP_ERR_CUDA, "building the symbol -> rows index failed");
    k_col_fill<<<rb, 256, 0, s>>>(P->d_fullOff, P->d_fullIdx, P->n_rows, cnt, rows);
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(SP_ERR_CUDA, "building the symbol -> rows index failed");
    dev_free(cnt);
    P->d_colFullOff = off;
    P->d_colFullRows = rows;
    return SP_OK;
}

// Records start from their rows' constants (the push path XORs into them).
// Word-major: word w of row j at rec[w * nrows + j].
__global__ void __launch_bounds__(256) k_rec_init(const uint8_t *__restrict__ cst, int64_t nrows, int64_t nwords,
                                                  uint32_t *rec)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows * nwords) return;
    rec[i] = cst[i % nrows] ? FULLM : 0u;
}

// K5 for nwords 32-shot words: the parent chains (one warp per 1024 shots
// walking every row in order) where there are enough such warps to fill the
// GPU, else every row at once from its full symbol list (when the program
// kept it).
static sp_status launch_gather(const sp_program *P, const uint32_t *B, int64_t pitch, int64_t nwords, uint32_t *recT,
                               cudaStream_t s)
{
    const int64_t warps = ceil_div(nwords, 32);
    if (P->d_fullIdx && warps < 4 * 152) {
        const int64_t all = warps * P->n_rows;
        k_gather_full<<<(unsigned)ceil_div(all, 8), 256, 0, s>>>(B, pitch, nwords, P->d_fullOff, P->d_fullIdx,
                                                                 P->d_const, P->n_rows, recT, pitch);
    } else {
        k_gather<<<(unsigned)ceil_div(warps, 4), 128, 0, s>>>(B, pitch, nwords, P->d_rowOff, P->d_idx, P->d_parent,
                                                                P->d_cflag, P->n_rows, recT, pitch);
    }
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

// The same three launches as sample_chunk, on caller-provided scratch:
// B (n_sym rows) and recT (n_rows rows), both with `pitch` 32-shot words per
// row; nshots must not exceed 32 * pitch.  Used by the entry point that
// allocates nothing.
sp_status sample_chunk_into(const sp_program *P, uint32_t *B, uint32_t *recT, int64_t pitch,
                            uint64_t seed, uint64_t shot0, uint64_t nshots, uint64_t *d_meas,
                            uint64_t *d_det, uint64_t *d_obs, cudaStream_t s)
{
    if (nshots == 0) return SP_OK;
    const int64_t nwords = (int64_t)((nshots + 31) / 32);
    if (nwords > pitch) return set_error(SP_ERR_INVALID_ARG, "chunk larger than the scratch pitch");
    if (P->n_sym > 0) {
        sp_status st = launch_draw_staged(P, seed, shot0, nwords, B, pitch, s);
        if (st != SP_OK) return st;
    }
    if (P->n_rows > 0) SP_TRY(launch_gather(P, B, pitch, nwords, recT, s));
    struct Seg { uint64_t *dst; int64_t row0, n; } segs[3] = {
        {d_meas, 0, P->n_meas}, {d_det, P->n_meas, P->n_det}, {d_obs, P->n_meas + P->n_det, P->n_obs}};
    for (const Seg &g : segs) {
        if (!g.dst || g.n == 0) continue;
        const int64_t words32 = 2 * ceil_div(g.n, 64);
        dim3 grid((unsigned)ceil_div(nwords, 8), (unsigned)ceil_div(words32 * 32, 256));
        k_emit<<<grid, 256, 0, s>>>(recT, pitch, 1, g.row0, g.n, (int64_t)nshots,
                                    reinterpret_cast<uint32_t *>(g.dst), words32);
        SP_CUDA(cudaGetLastError());
    }
    return SP_OK;
}

int64_t default_chunk(const sp_program *P)
{
    const double per_shot = (double)(P->n_sym + P->n_rows) / 8.0 + 64.0;
    const double budget = 4.0e9;
    int64_t c = (int64_t)(budget / per_shot);
    c = std::min<int64_t>(c, (int64_t)1 << 20);
    c = std::max<int64_t>(1024, (c / 1024) * 1024);
    return c;
}

sp_status ensure_scratch(sp_program *P, size_t shots)
{
    if (P->scratch_shots >= shots && P->d_B && P->d_recT) return SP_OK;
    dev_free(P->d_B);
    dev_free(P->d_recT);
    P->d_B = nullptr;
    P->d_recT = nullptr;
    P->scratch_shots = 0;
    const size_t words = (shots + 31) / 32;
    const size_t bsz = (size_t)std::max<int64_t>(P->n_sym, 1) * words * 4;
    const size_t rsz = (size_t)std::max<int64_t>(P->n_rows, 1) * words * 4;
    if (dev_alloc((void **)&P->d_B, bsz) != cudaSuccess) {
        cudaGetLastError();
        P->d_B = nullptr;
        return set_error(SP_ERR_OOM, "cudaMalloc of the fault-bit scratch failed");
    }
    if (dev_alloc((void **)&P->d_recT, rsz) != cudaSuccess) {
        cudaGetLastError();
        dev_free(P->d_B);
        P->d_B = nullptr;
        P->d_recT = nullptr;
        return set_error(SP_ERR_OOM, "cudaMalloc of the record scratch failed");
    }
    P->scratch_shots = words * 32;
    return SP_OK;
}

sp_status sample_chunk(sp_program *P, uint64_t seed, uint64_t shot0, uint64_t nshots,
                       uint64_t *d_meas, uint64_t *d_det, uint64_t *d_obs, cudaStream_t s)
{
    if (nshots == 0) return SP_OK;
    const int64_t nwords = (int64_t)((nshots + 31) / 32);
    const int64_t pitch = (int64_t)((P->scratch_shots + 31) / 32);
    if (P->path == SP_PATH_FUSED && P->fused_tw)
        return fused_chunk(P, seed, shot0, nshots, d_meas, d_det, d_obs, s);
    if (P->path == SP_PATH_DENSE || P->path == SP_PATH_TENSOR)
        return dense_chunk(P, seed, shot0, nshots, d_meas, d_det, d_obs, s);
    const int64_t warps = ceil_div(nwords, 32);
    int64_t rstride = pitch, wstride = 1;   // the records' layout (row-major unless pushed)
    if (P->d_fullIdx && P->n_sym > 0 && P->n_rows > 0 && warps < 4 * 152 &&
        (uint64_t)P->n_rows * (uint64_t)nwords * 4u <= PUSH_MAX_BYTES && P->n_blk < PUSH_MAX_BLOCKS) {
        // few shots and records that fit in L2: fired symbols go straight
        // into the records (no fault-bit table); the records are word-major
        // here, so that the warps of neighbouring shots XOR into different
        // L2 lines of a row (row-major, 16 of them shared each line and the
        // atomics serialised on it: 14.4 ms instead of 9.3 ms on Fig. 3c at
        // n = 1,000)
        SP_TRY(ensure_colfull(P, s));
        ProfScope ps(P, SP_KERNEL_DRAW, s);
        k_rec_init<<<(unsigned)ceil_div(P->n_rows * nwords, 256), 256, 0, s>>>(P->d_const, P->n_rows, nwords,
                                                                               P->d_recT);
        SP_CUDA(cudaGetLastError());
        SP_TRY(launch_draw_push(P, seed, shot0, nwords, P->d_recT, s));
        rstride = 1;
        wstride = P->n_rows;
    } else {
        if (P->n_sym > 0) {
            ProfScope ps(P, SP_KERNEL_DRAW, s);
            sp_status st = launch_draw_staged(P, seed, shot0, nwords, P->d_B, pitch, s);
            if (st != SP_OK) return st;
        }
        if (P->n_rows > 0) {
            ProfScope ps(P, SP_KERNEL_PRODUCT, s);
            SP_TRY(launch_gather(P, P->d_B, pitch, nwords, P->d_recT, s));
        }
    }
    struct Seg { uint64_t *dst; int64_t row0, n; } segs[3] = {
        {d_meas, 0, P->n_meas}, {d_det, P->n_meas, P->n_det}, {d_obs, P->n_meas + P->n_det, P->n_obs}};
    for (const Seg &g : segs) {
        if (!g.dst || g.n == 0) continue;
        const int64_t words32 = 2 * ceil_div(g.n, 64);
        dim3 grid((unsigned)ceil_div(nwords, 8), (unsigned)ceil_div(words32 * 32, 256));
        ProfScope ps(P, SP_KERNEL_EMIT, s);
        k_emit<<<grid, 256, 0, s>>>(P->d_recT, rstride, wstride, g.row0, g.n, (int64_t)nshots,
                                    reinterpret_cast<uint32_t *>(g.dst), words32);
        SP_CUDA(cudaGetLastError());
    }
    return SP_OK;
}

}  // namespace sp
