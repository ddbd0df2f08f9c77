// sp_dense.cu -- the dense forms of the sampler's product (Eq. sampling):
// rec_j(shot) = parity(<A_j, b_shot>) with b_0 = 1, taken as a contraction
// over all symbols instead of over the nonzero ones.  They pay where the
// coefficient rows are dense (the random layered circuits of Sec. 5, Fig. 3),
// not for surface codes.
//
//   k_popc_product  CUDA cores: per (row, 32 shots) the XOR of (A_j & b)
//                   over the row's words, then popcount parity;
//   k_tc_product    tensor cores (tcgen05): the 0/1 matrices as FP8 E4M3
//                   operands, exact FP32 accumulation (a sum of at most
//                   n_s + 1 < 2^24 ones), parity of the integer result.
//
// Both read the fault bits drawn shot-major by k_draw_dense (Philox stream
// identical to every other path) and the coefficient words transposed once
// per program (d_AT), and write the shot-major packed records directly.
#include <algorithm>

#include "sp_internal.h"

namespace sp {

namespace {

// AT[w][r] = A[r][w] for r < n_rows, 0 for the padding rows up to rpitch.
__global__ void k_transpose_words(const uint32_t *__restrict__ A, int64_t apitch, int64_t n_rows,
                                  uint32_t *__restrict__ AT, int64_t rpitch)
{
    __shared__ uint32_t t[32][33];
    const int64_t w0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    for (int k = ty; k < 32; k += 8) {
        const int64_t r = r0 + k, w = w0 + tx;
        t[k][tx] = (r < n_rows && w < apitch) ? A[(size_t)r * apitch + w] : 0u;
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int64_t w = w0 + k, r = r0 + tx;
        if (w < apitch && r < rpitch) AT[(size_t)w * rpitch + r] = t[tx][k];
    }
}

constexpr int POPC_KC = 128;   // fault-bit words of a 32-shot group staged per pass (16 KB)

// Warp = 32 consecutive rows of one record kind (lane = row), CTA = 8 warps,
// blockIdx.x = group of 32 shots.  acc[s] collects A_j & b for shot s word by
// word; the parity of its popcount is the record.  A warp transpose turns the
// 32 rows x 32 shots bits into one 32-row word per shot.
__global__ void __launch_bounds__(256) k_popc_product(const uint32_t *__restrict__ Bd, int64_t bpitch,
                                                      const uint32_t *__restrict__ AT, int64_t rpitch,
                                                      int64_t row0, int64_t nrow, int64_t words32,
                                                      uint64_t nshots, uint32_t *__restrict__ out)
{
    __shared__ __align__(16) uint32_t Bs[POPC_KC * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t g = blockIdx.x;
    const int64_t q = (int64_t)blockIdx.y * 8 + warp;      // 32-row word within the record kind
    const int64_t r = q * 32 + lane;
    const bool live = q < words32;
    const bool valid = live && r < nrow;
    const uint32_t *a = AT + (row0 + (valid ? r : 0));
    const uint32_t *bsrc = Bd + (size_t)g * (size_t)bpitch * 32u;
    uint32_t acc[32];
#pragma unroll
    for (int s = 0; s < 32; s++) acc[s] = 0u;
    for (int64_t k0 = 0; k0 < bpitch; k0 += POPC_KC) {
        const int kc = (int)(bpitch - k0 < POPC_KC ? bpitch - k0 : POPC_KC);
        __syncthreads();
        const uint4 *src = reinterpret_cast<const uint4 *>(bsrc + (size_t)k0 * 32u);
        for (int i = threadIdx.x; i < kc * 8; i += blockDim.x) reinterpret_cast<uint4 *>(Bs)[i] = src[i];
        __syncthreads();
        if (live) {
            for (int w = 0; w < kc; w++) {
                const uint32_t av = valid ? a[(size_t)(k0 + w) * (size_t)rpitch] : 0u;
                const uint4 *bw = reinterpret_cast<const uint4 *>(Bs + w * 32);
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    const uint4 b = bw[j];
                    acc[4 * j + 0] ^= av & b.x;
                    acc[4 * j + 1] ^= av & b.y;
                    acc[4 * j + 2] ^= av & b.z;
                    acc[4 * j + 3] ^= av & b.w;
                }
            }
        }
    }
    if (!live) return;
    uint32_t x = 0;
#pragma unroll
    for (int s = 0; s < 32; s++) x |= (uint32_t)(__popc(acc[s]) & 1) << s;
    const uint32_t y = transpose32(x, lane);
    const uint64_t shot = (uint64_t)g * 32u + (uint64_t)lane;
    if (shot < nshots) out[shot * (uint64_t)words32 + (uint64_t)q] = y;
}

// ---------------------------------------------------------------------------
// Tensor-core product (tcgen05, kind::f8f6f4, E4M3 operands, FP32 in TMEM)
// ---------------------------------------------------------------------------
// Tile: M = 128 shots x N = 256 record rows of one record kind, K in stages of
// TC_KS = 192 symbols held in a ring of TC_NS = 3 stage buffers.  Operands are
// K-major with no swizzle, in 8-row x 16-byte core matrices; in a stage
// buffer the core matrix (row group rg, K group kg) sits at
// kg * LBO + rg * TC_SBO, LBO = (rows / 8) * 128 bytes.
constexpr int TC_M = 128, TC_N = 256, TC_KS = 192, TC_NS = 3;
constexpr int TC_EXPANDERS = 256, TC_THREADS = TC_EXPANDERS + 32;   // 8 expander warps + 1 issuer warp
constexpr uint32_t TC_ABYTES = TC_M * TC_KS;                       // 16 KB: shots x symbols
constexpr uint32_t TC_BBYTES = TC_N * TC_KS;                       // 32 KB: rows x symbols
constexpr uint32_t TC_SBO = 128, TC_ALBO = (TC_M / 8) * 128, TC_BLBO = (TC_N / 8) * 128;
constexpr int TC_KG = TC_KS / 16;                                    // K groups per stage
constexpr uint32_t TC_TMEM_COLS = TC_N;
constexpr uint64_t TC_WAIT_NS = 2000000000ull;   // 2 s: default bound on the stage waits, and the drain's bound
constexpr uint32_t E4M3_ONE = 0x38u;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0u;
}

// Wait for the phase with the given parity to complete, for at most
// limit_ns; false if the bound ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets in 16-byte units, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f8f6f4: D in FP32, A and B E4M3, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t TC_IDESC = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(TC_IDESC), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 16 bits (element e = bit e) to 16 E4M3 bytes, 1.0 for a set bit: each
// nibble is spread to the low bits of four bytes by one product.
__device__ __forceinline__ uint4 bits16_to_e4m3(uint32_t h)
{
    uint4 r;
    r.x = (((h & 15u) * 0x00204081u) & 0x01010101u) * E4M3_ONE;
    r.y = ((((h >> 4) & 15u) * 0x00204081u) & 0x01010101u) * E4M3_ONE;
    r.z = ((((h >> 8) & 15u) * 0x00204081u) & 0x01010101u) * E4M3_ONE;
    r.w = ((((h >> 12) & 15u) * 0x00204081u) & 0x01010101u) * E4M3_ONE;
    return r;
}

__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// The coefficient rows of one record kind as tile-ready E4M3 stage blocks:
// block (tile, ks) holds rows tile*TC_N.. of the kind and symbols (with s_0)
// ks*TC_KS.., in the stage-buffer layout; rows past the kind and symbols past
// the row are zero.
__global__ void k_coef_e4m3(const uint32_t *__restrict__ A, int64_t apitch, int64_t row0, int64_t nrow,
                            int64_t ntiles, int64_t nks, uint4 *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per_block = TC_BBYTES / 16;
    if (i >= ntiles * nks * per_block) return;
    const int64_t blk = i / per_block;
    const uint32_t c = (uint32_t)(i % per_block);   // byte offset c*16 = kg*LBO + rg*SBO + r8*16
    const int64_t tile = blk / nks, ks = blk % nks;
    const uint32_t kg = c / TC_N, rg = (c >> 3) % (TC_N / 8), r8 = c & 7u;
    const int64_t r = tile * TC_N + rg * 8 + r8;
    const int64_t w = ks * (TC_KS / 32) + (kg >> 1);
    uint32_t h = 0;
    if (r < nrow && w < apitch) h = (A[(size_t)(row0 + r) * (size_t)apitch + (size_t)w] >> ((kg & 1u) * 16u)) & 0xFFFFu;
    out[i] = bits16_to_e4m3(h);
}

// Grid: x = tile of TC_M = 128 shots, y = tile of TC_N = 256 rows of one
// record kind.
// Warp specialised, synchronised by per-stage mbarriers instead of CTA
// barriers: warps 0-7 (expanders) turn the shots' fault bits, loaded one
// stage ahead into registers, into the E4M3 operand of each stage and
// arrive on its afull barrier; lane 0 of warp 8 (issuer) keeps the
// coefficient blocks of the next TC_NS-1 stages in flight (bulk copies on
// the full barriers), waits for both operands of a stage, issues TC_KS/32
// MMAs of K = 32 into the TMEM accumulator (128 lanes = shots x TC_N
// columns = rows, held by warp 8) and commits them to the stage's done
// barrier, which frees the stage's buffers.  The epilogue (warps 0-7) reads
// the exact FP32 counts and keeps their parity.  Every wait is bounded; a
// timeout raises the CTA's abort flag, every loop stops at its next check,
// the issuer drains its own copies and MMAs (again bounded), status 1 is
// recorded and TMEM is freed.  wait_ns bounds the stage waits (tests shorten
// it to make them run out); the drain of copies and MMAs already issued
// keeps the fixed bound TC_WAIT_NS, since they must land before TMEM is
// freed and the CTA exits.
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_product(const uint32_t *__restrict__ Bd, int64_t bpitch, int64_t ngroups, const uint4 *__restrict__ coef,
                 int64_t nks, int64_t words32, uint64_t nshots, uint32_t *__restrict__ out, int *status,
                 uint64_t wait_ns)
{
    extern __shared__ uint8_t smraw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    uint8_t *Abuf = sm;                                        // TC_NS stage buffers
    uint8_t *Bbuf = sm + TC_NS * TC_ABYTES;                    // TC_NS stage buffers
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + TC_NS * (TC_ABYTES + TC_BBYTES));   // full, afull, done [NS]
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bars + 3 * TC_NS);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool issuer_warp = warp == TC_EXPANDERS / 32;
    const int64_t m0 = (int64_t)blockIdx.x * TC_M;
    const int64_t nt = blockIdx.y;
    const uint32_t full = smem_u32(&bars[0]), afull = smem_u32(&bars[TC_NS]), done = smem_u32(&bars[2 * TC_NS]);
    if (tid == 0) {
        for (int i = 0; i < TC_NS; i++) {
            mbar_init(full + 8 * i, 1);
            mbar_init(afull + 8 * i, TC_EXPANDERS);
            mbar_init(done + 8 * i, 1);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (issuer_warp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;
    bool failed = false;
    int64_t issued = 0, copied = 0, landed = 0;   // issuer's progress
    if (!issuer_warp) {
        // ---- expanders: shot m of the tile, K groups kgb .. kgb+TC_KG/2-1 of each stage
        const int m = tid & (TC_M - 1);
        const uint32_t kgb = (uint32_t)(tid >> 7) * (TC_KG / 2);
        const int64_t g = (m0 + m) / 32;
        const bool mvalid = g < ngroups;
        const uint32_t *bsrc = Bd + (size_t)(mvalid ? g : 0) * (size_t)bpitch * 32u + (m & 31);
        const uint32_t a_off = (uint32_t)(m >> 3) * TC_SBO + (uint32_t)(m & 7) * 16u;
        constexpr int NW = TC_KG / 4;   // fault-bit words this thread expands per stage
        uint32_t vn[NW];
        auto load_words = [&](int64_t ks) {
#pragma unroll
            for (int j = 0; j < NW; j++) {
                const int64_t w = ks * (TC_KS / 32) + (kgb >> 1) + j;
                vn[j] = (mvalid && w < bpitch) ? bsrc[(size_t)w * 32u] : 0u;
            }
        };
        load_words(0);
        for (int64_t ks = 0; ks < nks; ks++) {
            if (*abort_flag) break;
            const int b = (int)(ks % TC_NS);
            // the MMAs of stage ks - TC_NS read this buffer last
            if (ks >= TC_NS && !mbar_wait(done + 8 * b, (uint32_t)(((ks / TC_NS) - 1) & 1), wait_ns)) {
                failed = true;
                *abort_flag = 1;
                break;
            }
            uint32_t v[NW];
#pragma unroll
            for (int j = 0; j < NW; j++) v[j] = vn[j];
            if (ks + 1 < nks) load_words(ks + 1);
            uint8_t *Ab = Abuf + b * TC_ABYTES;
#pragma unroll
            for (int j = 0; j < NW; j++) {
                const uint32_t kg = kgb + 2u * (uint32_t)j;
                *reinterpret_cast<uint4 *>(Ab + kg * TC_ALBO + a_off) = bits16_to_e4m3(v[j] & 0xFFFFu);
                *reinterpret_cast<uint4 *>(Ab + (kg + 1u) * TC_ALBO + a_off) = bits16_to_e4m3(v[j] >> 16);
            }
            fence_proxy_async_smem();
            mbar_arrive(afull + 8 * b);
        }
    } else if (lane == 0) {
        // ---- issuer
        const uint4 *cblk = coef + (size_t)nt * (size_t)nks * (TC_BBYTES / 16);
        auto prefetch = [&](int64_t j) {
            const int jb = (int)(j % TC_NS);
            mbar_expect_tx(full + 8 * jb, TC_BBYTES);
            bulk_g2s(smem_u32(Bbuf + jb * TC_BBYTES), cblk + (size_t)j * (TC_BBYTES / 16), TC_BBYTES, full + 8 * jb);
            copied = j + 1;
        };
        for (int64_t j = 0; j < TC_NS - 1 && j < nks; j++) prefetch(j);
        for (int64_t ks = 0; ks < nks; ks++) {
            if (*abort_flag) break;
            const int b = (int)(ks % TC_NS);
            const uint32_t par = (uint32_t)((ks / TC_NS) & 1);
            if (!mbar_wait(afull + 8 * b, par, wait_ns) || !mbar_wait(full + 8 * b, par, wait_ns)) {
                failed = true;
                *abort_flag = 1;
                break;
            }
            landed = ks + 1;
            tc_fence_after();
            const uint32_t a0 = smem_u32(Abuf + b * TC_ABYTES), b0 = smem_u32(Bbuf + b * TC_BBYTES);
#pragma unroll
            for (int s = 0; s < TC_KS / 32; s++)
                tc_mma(tmem, smem_desc(a0 + (uint32_t)s * 2u * TC_ALBO, TC_ALBO, TC_SBO),
                       smem_desc(b0 + (uint32_t)s * 2u * TC_BLBO, TC_BLBO, TC_SBO), (ks > 0 || s > 0) ? 1u : 0u);
            tc_commit(done + 8 * b);
            issued = ks + 1;
            // stage ks + TC_NS - 1 reuses the buffers of stage ks - 1 once its MMAs are done;
            // the MMAs of stage ks keep the tensor pipe busy meanwhile
            const int64_t j = ks + TC_NS - 1;
            if (j < nks) {
                if (ks >= 1 &&
                    !mbar_wait(done + 8 * (int)((ks - 1) % TC_NS), (uint32_t)(((ks - 1) / TC_NS) & 1), wait_ns)) {
                    failed = true;
                    *abort_flag = 1;
                    break;
                }
                prefetch(j);
            }
        }
        // drain: the last committed stage covers every MMA before it
        if (issued > 0) {
            const int64_t last = issued - 1;
            if (!mbar_wait(done + 8 * (int)(last % TC_NS), (uint32_t)((last / TC_NS) & 1), TC_WAIT_NS)) failed = true;
        }
        for (int64_t j = landed; j < copied; j++)
            if (!mbar_wait(full + 8 * (int)(j % TC_NS), (uint32_t)((j / TC_NS) & 1), TC_WAIT_NS)) failed = true;
        if (issued != nks) failed = true;
    }
    const bool all_ok = !__syncthreads_or(failed || *abort_flag);
    if (all_ok && !issuer_warp) {
        tc_fence_after();
        // warp: TMEM lanes 32*qw.. (its shots), columns (rows) half*TC_N/2..
        const int qw = warp & 3, half = warp >> 2;
        const uint32_t taddr = tmem + ((uint32_t)(32 * qw) << 16) + (uint32_t)(half * (TC_N / 2));
        const uint64_t shot = (uint64_t)m0 + (uint64_t)(32 * qw + lane);
#pragma unroll
        for (int c = 0; c < TC_N / 64; c++) {
            uint32_t v[32];
            tc_ld32(taddr + 32u * (uint32_t)c, v);
            uint32_t word = 0;
#pragma unroll
            for (int k = 0; k < 32; k++) word |= (__float2uint_rz(__uint_as_float(v[k])) & 1u) << k;
            const int64_t q = nt * (TC_N / 32) + half * (TC_N / 64) + c;
            if (shot < nshots && q < words32) out[shot * (uint64_t)words32 + (uint64_t)q] = word;
        }
    } else if (!all_ok && tid == 0) {
        atomicExch(status, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (issuer_warp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
}

// TC_NS stage buffers per operand, alignment, barriers and the TMEM address.
constexpr size_t TC_SMEM = TC_NS * (size_t)(TC_ABYTES + TC_BBYTES) + 1024 + 24 * TC_NS + 16;

}  // namespace

sp_status ensure_dense(sp_program *P, size_t shots, cudaStream_t s)
{
    if (!P->d_AT) {
        P->rpitch = ceil_div(std::max<int64_t>(P->n_rows, 1), 32) * 32;
        if (dev_alloc((void **)&P->d_AT, (size_t)P->apitch * (size_t)P->rpitch * 4) != cudaSuccess) {
            cudaGetLastError();
            P->d_AT = nullptr;
            return set_error(SP_ERR_OOM, "cudaMalloc of the transposed coefficient words failed");
        }
        dim3 grid((unsigned)ceil_div(P->apitch, 32), (unsigned)(P->rpitch / 32));
        k_transpose_words<<<grid, dim3(32, 8), 0, s>>>(P->d_A, P->apitch, P->n_rows, P->d_AT, P->rpitch);
        SP_CUDA(cudaGetLastError());
    }
    if (P->dense_shots < shots || !P->d_Bd) {
        dev_free(P->d_Bd);
        P->d_Bd = nullptr;
        P->dense_shots = 0;
        const size_t groups = (shots + 31) / 32;
        if (dev_alloc((void **)&P->d_Bd, groups * (size_t)P->apitch * 32u * 4u) != cudaSuccess) {
            cudaGetLastError();
            P->d_Bd = nullptr;
            return set_error(SP_ERR_OOM, "cudaMalloc of the shot-major fault-bit scratch failed");
        }
        P->dense_shots = groups * 32;
    }
    return SP_OK;
}

bool tensor_path_available(const sp_program *P)
{
    int major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, P->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, P->device) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    // sums of at most apitch*32 ones stay exact in FP32 below 2^24
    return major == 10 && minor == 3 && P->n_rows > 0 && P->n_sym > 0 && P->apitch * 32 < (int64_t)1 << 24;
}

// E4M3 stage blocks of the coefficient rows, per record kind, and the
// device status word of the tensor-core kernel.
static sp_status ensure_tensor(sp_program *P, cudaStream_t s)
{
    if (P->tc_ready) return SP_OK;
    const int64_t rows0[3] = {0, P->n_meas, P->n_meas + P->n_det};
    const int64_t nrow[3] = {P->n_meas, P->n_det, P->n_obs};
    P->tc_nks = ceil_div(P->apitch, TC_KS / 32);
    for (int k = 0; k < 3; k++) {
        P->tc_ntiles[k] = nrow[k] ? ceil_div(2 * ceil_div(nrow[k], 64), TC_N / 32) : 0;
        dev_free(P->d_tc_coef[k]);
        P->d_tc_coef[k] = nullptr;
        if (!P->tc_ntiles[k]) continue;
        const int64_t chunks = P->tc_ntiles[k] * P->tc_nks * (TC_BBYTES / 16);
        if (dev_alloc((void **)&P->d_tc_coef[k], (size_t)chunks * 16) != cudaSuccess) {
            cudaGetLastError();
            P->d_tc_coef[k] = nullptr;
            return set_error(SP_ERR_OOM, "cudaMalloc of the tensor-core coefficient blocks failed");
        }
        k_coef_e4m3<<<(unsigned)ceil_div(chunks, 256), 256, 0, s>>>(P->d_A, P->apitch, rows0[k], nrow[k],
                                                                    P->tc_ntiles[k], P->tc_nks,
                                                                    reinterpret_cast<uint4 *>(P->d_tc_coef[k]));
        SP_CUDA(cudaGetLastError());
    }
    if (!P->d_tc_status) {
        int *st = nullptr;
        if (dev_alloc((void **)&st, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return set_error(SP_ERR_OOM, "cudaMalloc of the device status word failed");
        }
        SP_CUDA(cudaMemsetAsync(st, 0, sizeof(int), s));
        P->d_tc_status = st;
    }
    SP_CUDA(cudaFuncSetAttribute(k_tc_product, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
    P->tc_ready = true;
    return SP_OK;
}

sp_status dense_chunk(sp_program *P, uint64_t seed, uint64_t shot0, uint64_t nshots, uint64_t *d_meas,
                      uint64_t *d_det, uint64_t *d_obs, cudaStream_t s)
{
    if (nshots == 0) return SP_OK;
    sp_status st = ensure_dense(P, (size_t)nshots, s);
    if (st != SP_OK) return st;
    const int64_t groups = (int64_t)((nshots + 31) / 32);
    {
        ProfScope ps(P, SP_KERNEL_DRAW, s);
        if ((st = launch_draw_dense(P, seed, shot0, groups, P->d_Bd, P->apitch, s)) != SP_OK) return st;
    }
    struct Seg { uint64_t *dst; int64_t row0, n; } segs[3] = {
        {d_meas, 0, P->n_meas}, {d_det, P->n_meas, P->n_det}, {d_obs, P->n_meas + P->n_det, P->n_obs}};
    if (P->path == SP_PATH_TENSOR) {
        if ((st = ensure_tensor(P, s)) != SP_OK) return st;
        for (int k = 0; k < 3; k++) {
            const Seg &g = segs[k];
            if (!g.dst || g.n == 0) continue;
            const int64_t words32 = 2 * ceil_div(g.n, 64);
            ProfScope ps(P, SP_KERNEL_TENSOR, s);
            dim3 grid((unsigned)ceil_div((int64_t)nshots, TC_M), (unsigned)P->tc_ntiles[k]);
            k_tc_product<<<grid, TC_THREADS, TC_SMEM, s>>>(P->d_Bd, P->apitch, groups,
                                                          reinterpret_cast<const uint4 *>(P->d_tc_coef[k]), P->tc_nks,
                                                          words32, nshots, reinterpret_cast<uint32_t *>(g.dst),
                                                          P->d_tc_status, P->tc_wait_ns ? P->tc_wait_ns : TC_WAIT_NS);
            SP_CUDA(cudaGetLastError());
        }
        return SP_OK;
    }
    for (const Seg &g : segs) {
        if (!g.dst || g.n == 0) continue;
        const int64_t words32 = 2 * ceil_div(g.n, 64);
        ProfScope ps(P, SP_KERNEL_PRODUCT, s);
        dim3 grid((unsigned)groups, (unsigned)ceil_div(words32, 8));
        k_popc_product<<<grid, 256, 0, s>>>(P->d_Bd, P->apitch, P->d_AT, P->rpitch, g.row0, g.n, words32, nshots,
                                            reinterpret_cast<uint32_t *>(g.dst));
        SP_CUDA(cudaGetLastError());
    }
    return SP_OK;
}

}  // namespace sp

namespace sp {

namespace {

sp_status run_path(sp_program *P, uint64_t seed, uint64_t shot0, uint64_t shots, uint64_t *om, uint64_t *od,
                   uint64_t *oo, cudaStream_t s)
{
    const int64_t wm = (P->n_meas + 63) / 64, wd = (P->n_det + 63) / 64, wo = (P->n_obs + 63) / 64;
    for (uint64_t done = 0; done < shots;) {
        const uint64_t n = std::min<uint64_t>(shots - done, (uint64_t)P->chunk_shots);
        sp_status st = sample_chunk(P, seed, shot0 + done, n, om + done * wm, od + done * wd, oo + done * wo, s);
        if (st != SP_OK) return st;
        done += n;
    }
    return SP_OK;
}

void drop_dense_buffers(sp_program *P)
{
    dev_free(P->d_Bd);
    dev_free(P->d_AT);
    for (auto &c : P->d_tc_coef) { dev_free(c); c = nullptr; }
    P->tc_ready = false;
    P->d_Bd = nullptr;
    P->d_AT = nullptr;
    P->dense_shots = 0;
}

}  // namespace

// Per-circuit choice of the product form.  The sparse form (the fused kernel
// when the records of a tile fit in shared memory, else the staged kernels)
// is the default; where at least 1 % of the coefficients are nonzero the
// two dense forms (AND/popcount, tensor cores) are also run on a probe of
// 32,768 shots (best of two timed runs after a warm-up) and the fastest is
// kept, the default unless another is at least 3 % faster.  Buffers of the
// forms not kept are released.
sp_status choose_path(sp_program *P, cudaStream_t s)
{
    P->build_path = P->fused_tw ? SP_PATH_FUSED : SP_PATH_SPARSE;
    P->path = P->build_path;
    for (double &t : P->path_probe_ms) t = 0.0;
    if (P->density < 0.01 || P->n_rows == 0 || P->n_sym == 0) return SP_OK;
    std::vector<int> cand{P->build_path, SP_PATH_DENSE};
    if (tensor_path_available(P)) cand.push_back(SP_PATH_TENSOR);
    const uint64_t shots = 32768;
    const int64_t words = (P->n_meas + 63) / 64 + (P->n_det + 63) / 64 + (P->n_obs + 63) / 64;
    uint64_t *out = nullptr;
    if (dev_alloc((void **)&out, (size_t)shots * (size_t)std::max<int64_t>(words, 1) * 8) != cudaSuccess) {
        cudaGetLastError();
        return set_error(SP_ERR_OOM, "cudaMalloc of the path probe outputs failed");
    }
    uint64_t *om = out, *od = om + shots * ((P->n_meas + 63) / 64), *oo = od + shots * ((P->n_det + 63) / 64);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool prof = P->profiling;
    P->profiling = false;
    sp_status st = SP_OK;
    int pick = P->build_path;
    float best = 1e30f;
    for (size_t ci = 0; ci < cand.size() && st == SP_OK; ci++) {
        P->path = cand[ci];
        if (uses_staged_scratch(P) && (st = ensure_scratch(P, (size_t)std::min<uint64_t>(shots, P->chunk_shots))) != SP_OK)
            break;
        if ((st = run_path(P, 1, 0, shots, om, od, oo, s)) != SP_OK) break;
        float ms = 1e30f;
        for (int rep = 0; rep < 2 && st == SP_OK; rep++) {
            cudaEventRecord(e0, s);
            st = run_path(P, 1, shots * (rep + 1), shots, om, od, oo, s);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) { st = cuda_error(cudaGetLastError(), "path probe"); break; }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            ms = std::min(ms, t);
        }
        if (st != SP_OK) break;
        if (cand[ci] == SP_PATH_TENSOR) {
            int32_t bad = 0;
            st = sp_device_status(P, &bad);
            if (st == SP_ERR_TIMEOUT) { st = SP_OK; continue; }   // a tile gave up on a bounded wait: never pick this form
            if (st != SP_OK) break;
        }
        P->path_probe_ms[cand[ci]] = ms;
        if (ci == 0 || ms < 0.97f * best) { best = ms; pick = cand[ci]; }
    }
    P->profiling = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dev_free(out);
    if (st != SP_OK) return st;
    P->build_path = pick;
    P->path = pick;
    if (pick != SP_PATH_DENSE && pick != SP_PATH_TENSOR) drop_dense_buffers(P);
    return SP_OK;
}

}  // namespace sp
