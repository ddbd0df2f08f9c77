// sp_internal.h -- internal declarations of the GB300 symbolic-phase library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "symphase.h"

namespace sp {

// ----------------------------------------------------------------------------
// Elementary instructions produced by flattening the circuit (one per target
// or target pair).  Detectors and observables do not appear here.
// ----------------------------------------------------------------------------
enum InstCode : uint32_t {
    I_H = 0, I_S, I_CX, I_X, I_Y, I_Z,
    I_M, I_MR, I_R,
    I_XERR, I_YERR, I_ZERR, I_DEP1, I_DEP2,
    I_XIF, I_YIF, I_ZIF    // feed-forward: a = qubit, b = record index
};

struct Inst {
    uint32_t code;
    uint32_t a;         // qubit
    uint32_t b;         // second qubit (CX, DEP2), record index (feed-forward)
    uint32_t aux;       // threshold T for noise ops
    uint32_t pbits;     // FP32 bits of the probability of noise ops
    uint32_t gi;        // noise ops: index among the circuit's noise ops
    uint32_t sym_base;  // noise ops: fault symbols before this one
    uint32_t pad;
};

// Channel kinds used by the draw kernel.
enum ChannelKind : uint8_t { CK_BERN = 0, CK_DEP1 = 1, CK_DEP2 = 2, CK_RANDOM = 3 };

// Events of the row-operation log written by the traversal's first pass and
// replayed column-parallel by the second (header = kind << 24 | count).
enum LogEvent : uint32_t {
    EV_INJECT = 1,   // [hdr|k, s0]            symbols s0..s0+k-1 get their injection columns
    EV_MRAND = 2,    // [hdr|cnt, p, s, rec, rows..]  random measurement with pivot p
    EV_MDET = 3,     // [hdr|cnt, rec, rows..]        deterministic measurement
    EV_RESET = 4,    // [hdr|cnt, rows..]             conditional X^e on the rows
    EV_FF = 5        // [hdr|cnt, rec, rows..]        rows ^= form of record rec (feed-forward)
};
constexpr uint32_t NO_REC = 0xFFFFFFFFu;

// Counters written by the traversal kernel.
struct TraverseCounts {
    uint64_t log_len;
    uint32_t nsym;
    uint32_t nch;
    uint32_t nrec;
    uint32_t err;      // 0 ok, 1 log overflow, 2 nondeterministic product phase
    uint32_t nev;      // events other than injections (their positions: ev_pos)
    uint32_t pad;
};

// ----------------------------------------------------------------------------
// A built program.
// ----------------------------------------------------------------------------
}  // namespace sp

struct sp_program {
    int device = 0;
    uint32_t n = 0;                 // qubits
    int64_t n_meas = 0, n_det = 0, n_obs = 0, n_rows = 0;
    int64_t n_sym = 0, n_ch = 0, n_rand = 0;
    int64_t log_len = 0;
    int64_t apitch = 0;             // u32 words per coefficient row
    // coefficient rows: meas, det, obs (bit 0 = constant)
    uint32_t *d_A = nullptr;
    // channels
    uint32_t *d_chT = nullptr;
    uint8_t *d_chKind = nullptr;
    float *d_chP = nullptr;         // circuit probabilities (FP32)
    uint32_t *d_chSym0 = nullptr;   // first symbol of each channel
    // sparse sampler program: row j = parent (or none) XOR const XOR sum of B rows
    uint32_t *d_rowOff = nullptr;   // [n_rows+1]
    uint32_t *d_idx = nullptr;      // symbol-1 indices
    // full rows (symbol-1 indices of A_j, constant excluded), kept when at
    // most FULL_ROWS_KEEP entries: the row-parallel product for few shots
    uint32_t *d_fullOff = nullptr;  // [n_rows+1]
    uint32_t *d_fullIdx = nullptr;
    // the same full rows by symbol: rows d_colFullRows[off[s] .. off[s+1]) hold symbol s+1
    uint32_t *d_colFullOff = nullptr;   // [n_sym+1]
    uint32_t *d_colFullRows = nullptr;
    int32_t *d_parent = nullptr;    // [n_rows]
    uint8_t *d_cflag = nullptr;     // [n_rows]
    int64_t nnz_rows = 0, nnz_delta = 0;
    // dense program: A rows in u64 words over symbols 1..n_s (bit s-1)
    uint64_t *d_A64 = nullptr;
    int64_t a64pitch = 0;
    uint8_t *d_const = nullptr;     // [n_rows]
    // expectation: row x channel incidence (bits) and its transpose
    uint32_t *d_inc = nullptr;      // [n_tgt][incPitch]
    uint32_t *d_incT = nullptr;     // [n_ch][incTPitch]
    int64_t incPitch = 0, incTPitch = 0;
    float *d_kappa = nullptr;       // [n_ch]
    float *d_wbuf = nullptr;        // [3 * n_ch] channel weights, derivatives, sign classes
    // scratch (owned, reused across sample calls)
    uint32_t *d_B = nullptr;        // fault bits, bit-sliced: [n_sym][chunk/32]
    uint32_t *d_recT = nullptr;     // records, bit-sliced: [n_rows][chunk/32]
    uint32_t *d_Bd = nullptr;       // dense paths: fault bits shot-major, [group of 32 shots][apitch][32]
    size_t dense_shots = 0;         // shots d_Bd holds
    uint32_t *d_AT = nullptr;       // dense paths: coefficient words transposed, [apitch][rpitch]
    int64_t rpitch = 0;             // rows of d_AT (n_rows rounded up to 32)
    uint8_t *d_tc_coef[3] = {nullptr, nullptr, nullptr};  // tensor path: E4M3 stage blocks per record kind
    int64_t tc_ntiles[3] = {0, 0, 0};                     // 256-row tiles per record kind
    int64_t tc_nks = 0;                                   // 192-symbol K stages
    int *d_tc_status = nullptr;                           // tensor kernel status word (0 = ok)
    uint64_t tc_wait_ns = 0;                              // bound of the tensor kernel's stage waits (0 = 2 s)
    bool tc_ready = false;                                // d_tc_coef built for the current program
    double path_probe_ms[5] = {0, 0, 0, 0, 0};            // build-time probe per path (0 = not timed)
    size_t scratch_shots = 0;
    int64_t chunk_shots = 0;
    int path = SP_PATH_SPARSE;
    int build_path = SP_PATH_SPARSE;
    uint64_t gen = 0;               // configuration generation: bumped by sp_set_path / _fused_config / _chunk
    double build_ms = 0.0;
    double density = 0.0;
    // host-side copies used for host entry points and batching
    std::vector<uint8_t> h_const;
    // detector/observable definitions: target t = XOR of measurement rows
    // h_xrefs[h_xoff[t] .. h_xoff[t+1])
    std::vector<uint32_t> h_xoff, h_xrefs;
    // pinned host staging for sp_sample_host (allocated lazily)
    void *h_stage = nullptr;
    size_t h_stage_bytes = 0;
    uint64_t *d_out_stage = nullptr;
    size_t d_out_stage_bytes = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // draw descriptors: blocks of 4 channels (thresholds, kinds/offsets, first symbol)
    int64_t n_blk = 0;
    int64_t n_blk_live = 0;            // blocks with a channel that can fire and changes some record
    uint4 *d_blkT = nullptr;
    uint32_t *d_blkMeta = nullptr;
    uint32_t *d_blkSym0 = nullptr;
    uint32_t *d_blkFilt = nullptr;  // per block: all-thresholds-large flag or the largest threshold
    uint4 *d_blkConst = nullptr;    // per block: a launch's Philox constants (rewritten by every fused launch)
    // grouped draw (stream 2, sp_grouped.cu): built on the first sp_set_stream(prog, 2)
    int stream = 1;
    std::vector<double> h_fault_p;    // probability of each channel other than random outcomes, in order
    uint4 *d_s2Ch = nullptr;
    uint4 *d_s2G = nullptr;
    uint32_t *d_s2Rand = nullptr;
    int64_t s2_nfault = 0, s2_ngrp = 0, s2_nrnd = 0;
    int s2_ctas_per_sm = 0, s2_cfg = 0;   // occupancy of the grouped kernel for launch shape s2_cfg
    // fused product program (see sp_fused.cu)
    uint8_t *d_fCflag = nullptr;      // step 0: constant bit of each measurement row's own part
    uint2 *d_fChain = nullptr;        // step B items (row, parent), per thread, parents first
    uint32_t *d_fBOff = nullptr;      // [threads+1]
    uint32_t *d_fCOff = nullptr;      // step C: target t = XOR of measurement rows d_fCRefs[off[t]..off[t+1])
    uint32_t *d_fCRefs = nullptr;
    // symbol -> measurement rows whose own part holds it (CSC of the own parts)
    uint32_t *d_colOff = nullptr;     // [n_sym + 1]
    uint32_t *d_colRows = nullptr;    // [nnz_delta]
    int smem_max = 0;
    int fused_tw = 0;                 // shots per tile / 32 (0 = fused path off)
    int fused_unroll = 1;             // 2: the 64- or 128-shot variant with one CTA per SM
    int fused_threads = 512;          // threads per CTA of the selected variant
    size_t fused_smem = 0;            // dynamic shared memory of a launch (with the staged tables, if any)
    size_t fused_smem_base = 0;       // the same without the staged phase-2 tables
    uint32_t fused_tab_off = 0;       // word offset of the staged phase-2 tables (0 = not staged)
    bool fused_emit_once = false;     // phase 3 stages all record kinds before one copy-out
    int64_t fused_items = 0;          // parent-chain items (phase 2B)
    uint32_t fused_aux_off = 0;       // shared-memory words before the queue/stage region
    bool tuned = false;
    int autotune_launches = 0;        // fused-kernel launches made by the autotuner
    int fused_ctas_per_sm = 1;
    int num_sms = 0;
    // per-kernel event profiling (sp_profile_enable)
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
};

namespace sp {

// error plumbing (sp_capi.cu)
sp_status set_error(sp_status st, const std::string &msg);
sp_status cuda_error(cudaError_t e, const char *what);

#define SP_TRY(x) do { sp_status _s = (x); if (_s != SP_OK) return _s; } while (0)

#define SP_CUDA(call)                                                  \
    do {                                                               \
        cudaError_t _e = (call);                                       \
        if (_e != cudaSuccess) return ::sp::cuda_error(_e, #call);     \
    } while (0)

// Every device allocation of the library goes through dev_alloc / dev_free
// (sp_capi.cu): they count the allocations held and honour the allocation-
// failure hook of sp_debug_fail_alloc, which makes one chosen allocation
// fail as if the device were out of memory.  host_alloc_fails() is the same
// hook for the host-side program object.
cudaError_t dev_alloc(void **p, size_t bytes);
void dev_free(void *p);
bool host_alloc_fails();

// build (sp_build.cu).  finish_program derives the sampler program, the
// expectation tables, the fused-kernel program and the path choice from
// P->d_A and the channel table (the traversal's output).
sp_status build_program(const sp_circuit_desc *desc, cudaStream_t stream, sp_program *P);
sp_status finish_program(sp_program *P, cudaStream_t stream);
uint32_t threshold_of(double p);

// A row's parent (the earlier row its own part is coded against) lies at
// most PARENT_LOOKBACK rows before it.
constexpr int PARENT_LOOKBACK = 512;
// Largest full-row index list a program keeps (1 GiB of indices).
constexpr uint64_t FULL_ROWS_KEEP = 1ull << 28;

// saved programs (sp_serial.cu): save_program writes the blob (size only
// when buf is NULL), check_saved validates one on the host, load_program
// validates and rebuilds it on the current device.
sp_status save_program(const sp_program *P, void *buf, size_t cap, size_t *size);
sp_status check_saved(const void *buf, size_t size);
sp_status load_program(const void *buf, size_t size, cudaStream_t stream, sp_program *P);

// profiling: bracket one kernel launch with events when enabled
struct ProfScope {
    sp_program *P;
    int cls;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(sp_program *P_, int cls_, cudaStream_t s_);
    ~ProfScope();
};

// the staged sparse kernels' scratch (d_B, d_recT) is needed on that path only
inline bool uses_staged_scratch(const sp_program *P)
{
    return !(P->path == SP_PATH_FUSED && P->fused_tw) && P->path != SP_PATH_DENSE && P->path != SP_PATH_TENSOR;
}

// sampling (sp_sample.cu)
sp_status ensure_scratch(sp_program *P, size_t shots);
sp_status sample_chunk(sp_program *P, uint64_t seed, uint64_t shot0, uint64_t nshots,
                       uint64_t *d_meas, uint64_t *d_det, uint64_t *d_obs, cudaStream_t s);
// shots shot0 .. shot0+nshots-1 through the program's current path, in chunks
sp_status sample_range(sp_program *P, uint64_t seed, uint64_t shot0, uint64_t nshots,
                       uint64_t *d_meas, uint64_t *d_det, uint64_t *d_obs, cudaStream_t s);
int64_t default_chunk(const sp_program *P);
// dense paths (sp_dense.cu)
sp_status ensure_dense(sp_program *P, size_t shots, cudaStream_t s);
sp_status choose_path(sp_program *P, cudaStream_t s);
bool tensor_path_available(const sp_program *P);
sp_status dense_chunk(sp_program *P, uint64_t seed, uint64_t shot0, uint64_t nshots, uint64_t *d_meas,
                      uint64_t *d_det, uint64_t *d_obs, cudaStream_t s);
// rec: word-major records, word w of row j at rec[w * n_rows + j]
sp_status launch_draw_push(const sp_program *P, uint64_t seed, uint64_t shot0, int64_t nwords, uint32_t *rec,
                           cudaStream_t s);
sp_status launch_draw_dense(const sp_program *P, uint64_t seed, uint64_t shot0, int64_t ngroups, uint32_t *Bd,
                            int64_t bpitch, cudaStream_t s);
// fused path (sp_fused.cu)
sp_status build_fused_program(sp_program *P, cudaStream_t s);
sp_status fused_chunk(sp_program *P, uint64_t seed, uint64_t shot0, uint64_t nshots, uint64_t *d_meas,
                      uint64_t *d_det, uint64_t *d_obs, cudaStream_t s);
sp_status sample_batch(sp_program *const *progs, uint32_t n, const uint64_t *seeds, const uint64_t *nshots,
                       uint64_t *const *d_meas, uint64_t *const *d_det, uint64_t *const *d_obs, cudaStream_t s);
void batch_forget(const sp_program *P);
size_t batch_plan_count();
constexpr size_t BATCH_MAX_PLANS = 8;
sp_status fused_select(sp_program *P, int tw, int unroll);
// grouped draw (sp_grouped.cu)
sp_status ensure_grouped(sp_program *P, cudaStream_t s);
sp_status grouped_chunk(sp_program *P, uint64_t seed, uint64_t shot0, uint64_t nshots, uint64_t *d_meas,
                        uint64_t *d_det, uint64_t *d_obs, cudaStream_t s);
sp_status autotune(sp_program *P, cudaStream_t s);
sp_status launch_draw_staged(const sp_program *P, uint64_t seed, uint64_t shot0, int64_t nwords, uint32_t *B,
                             int64_t pitch, cudaStream_t s);
sp_status sample_chunk_into(const sp_program *P, uint32_t *B, uint32_t *recT, int64_t pitch,
                            uint64_t seed, uint64_t shot0, uint64_t nshots, uint64_t *d_meas,
                            uint64_t *d_det, uint64_t *d_obs, cudaStream_t s);

// expectation (sp_expect.cu)
sp_status expect_fwd(sp_program *P, const float *d_p, float *d_logE, cudaStream_t s);
sp_status expect_bwd(sp_program *P, const float *d_p, const float *d_g, float *d_grad, cudaStream_t s);
sp_status expect_sign(sp_program *P, const float *d_p, float *d_sign, cudaStream_t s);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// 32x32 bit transpose across a warp: lane j receives, as bit l, bit j of
// lane l's word.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane)
{
    constexpr uint32_t FULL = 0xffffffffu;
    const uint32_t m16 = 0x0000FFFFu, m8 = 0x00FF00FFu, m4 = 0x0F0F0F0Fu, m2 = 0x33333333u, m1 = 0x55555555u;
    uint32_t y;
    y = __shfl_xor_sync(FULL, x, 16); x = (lane & 16) ? ((x & ~m16) | ((y >> 16) & m16)) : ((x & m16) | ((y & m16) << 16));
    y = __shfl_xor_sync(FULL, x, 8);  x = (lane & 8) ? ((x & ~m8) | ((y >> 8) & m8)) : ((x & m8) | ((y & m8) << 8));
    y = __shfl_xor_sync(FULL, x, 4);  x = (lane & 4) ? ((x & ~m4) | ((y >> 4) & m4)) : ((x & m4) | ((y & m4) << 4));
    y = __shfl_xor_sync(FULL, x, 2);  x = (lane & 2) ? ((x & ~m2) | ((y >> 2) & m2)) : ((x & m2) | ((y & m2) << 2));
    y = __shfl_xor_sync(FULL, x, 1);  x = (lane & 1) ? ((x & ~m1) | ((y >> 1) & m1)) : ((x & m1) | ((y & m1) << 1));
    return x;
}

// Raise a kernel's dynamic shared-memory limit to the most the device
// allows next to its static shared memory.  The limit belongs to the kernel,
// not to a program, so it is never lowered for one program's needs.
template <typename F>
inline cudaError_t max_dynamic_smem(F *kernel)
{
    int dev = 0, opt = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&opt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes a;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, (const void *)kernel);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void *)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 opt - (int)a.sharedSizeBytes);
    return e;
}

}  // namespace sp
