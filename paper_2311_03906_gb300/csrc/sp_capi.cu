// sp_capi.cu -- the extern "C" entry points declared in include/symphase.h.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <memory>
#include <new>
#include <string>

#include "sp_internal.h"

namespace sp {

static thread_local std::string g_last_error;

// Allocation-failure hook: the allocation that finds the counter at zero
// fails, then the hook disarms (-1 = off).  Live allocation counts.
static std::atomic<int64_t> g_fail_after{-1};
static std::atomic<int64_t> g_live_dev{0}, g_live_host{0};

static bool hook_fires()
{
    int64_t v = g_fail_after.load();
    while (v >= 0) {
        if (g_fail_after.compare_exchange_weak(v, v - 1)) return v == 0;
    }
    return false;
}

cudaError_t dev_alloc(void **p, size_t bytes)
{
    *p = nullptr;
    if (hook_fires()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) g_live_dev++;
    else *p = nullptr;
    return e;
}

void dev_free(void *p)
{
    if (!p) return;
    cudaFree(p);
    g_live_dev--;
}

bool host_alloc_fails() { return hook_fires(); }

sp_status set_error(sp_status st, const std::string &msg)
{
    g_last_error = msg;
    return st;
}

sp_status cuda_error(cudaError_t e, const char *what)
{
    cudaGetLastError();
    return set_error(SP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

static void release(sp_program *P)
{
    if (!P) return;
    batch_forget(P);
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != P->device) cudaSetDevice(P->device);
    void *bufs[] = {P->d_A, P->d_chT, P->d_chKind, P->d_chP, P->d_chSym0, P->d_rowOff, P->d_idx, P->d_fullOff, P->d_fullIdx, P->d_colFullOff, P->d_colFullRows,
                    P->d_parent, P->d_cflag, P->d_A64, P->d_const, P->d_inc, P->d_incT, P->d_kappa,
                    P->d_wbuf, P->d_B, P->d_recT, P->d_Bd, P->d_out_stage, P->d_blkT, P->d_blkMeta, P->d_blkFilt, P->d_blkConst,
                    P->d_blkSym0, P->d_fCflag, P->d_fChain, P->d_fBOff, P->d_fCOff, P->d_fCRefs,
                    P->d_colOff, P->d_colRows, P->d_AT, P->d_tc_coef[0], P->d_tc_coef[1], P->d_tc_coef[2],
                    P->d_tc_status, P->d_s2Ch, P->d_s2G, P->d_s2Rand};
    for (void *b : bufs) if (b) dev_free(b);
    if (P->h_stage) cudaFreeHost(P->h_stage);
    for (cudaEvent_t e : P->ev_pool) cudaEventDestroy(e);
    for (auto &pe : P->ev_pending) { cudaEventDestroy(pe.second.first); cudaEventDestroy(pe.second.second); }
    for (cudaEvent_t &e : P->ev) if (e) cudaEventDestroy(e);
    if (P->copy_stream) cudaStreamDestroy(P->copy_stream);
    if (cur >= 0 && cur != P->device) cudaSetDevice(cur);
    delete P;
    g_live_host--;
}

static int64_t words64(int64_t n) { return (n + 63) / 64; }

static cudaEvent_t pool_event(sp_program *P)
{
    if (!P->ev_pool.empty()) {
        cudaEvent_t e = P->ev_pool.back();
        P->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

ProfScope::ProfScope(sp_program *P_, int cls_, cudaStream_t s_) : P(P_), cls(cls_), s(s_)
{
    if (!P->profiling) return;
    a = pool_event(P);
    b = pool_event(P);
    if (a) cudaEventRecord(a, s);
}

ProfScope::~ProfScope()
{
    if (!P->profiling || !a || !b) return;
    cudaEventRecord(b, s);
    P->ev_pending.push_back({cls, {a, b}});
}

static sp_status check_ptr(const void *p, const char *name)
{
    if (p && (reinterpret_cast<uintptr_t>(p) & 7u))
        return set_error(SP_ERR_INVALID_ARG, std::string(name) + " is not 8-byte aligned");
    return SP_OK;
}

sp_status sample_range(sp_program *P, uint64_t seed, uint64_t shot0, uint64_t nshots,
                       uint64_t *d_meas, uint64_t *d_det, uint64_t *d_obs, cudaStream_t s)
{
    if (nshots == 0) return SP_OK;
    if (P->path == SP_PATH_FUSED && P->fused_tw)
        return fused_chunk(P, seed, shot0, nshots, d_meas, d_det, d_obs, s);
    const int64_t chunk = P->chunk_shots;
    sp_status st;
    if (uses_staged_scratch(P)) {
        st = ensure_scratch(P, (size_t)std::min<uint64_t>(nshots, (uint64_t)chunk));
        if (st != SP_OK) return st;
    }
    const int64_t wm = words64(P->n_meas), wd = words64(P->n_det), wo = words64(P->n_obs);
    for (uint64_t done = 0; done < nshots;) {
        const uint64_t n = std::min<uint64_t>(nshots - done, (uint64_t)chunk);
        st = sample_chunk(P, seed, shot0 + done, n, d_meas ? d_meas + done * wm : nullptr,
                          d_det ? d_det + done * wd : nullptr, d_obs ? d_obs + done * wo : nullptr, s);
        if (st != SP_OK) return st;
        done += n;
    }
    return SP_OK;
}

// A configuration change makes every batch plan holding the program stale.
static void reconfigured(sp_program *P)
{
    P->gen++;
    batch_forget(P);
}

}  // namespace sp

using namespace sp;

extern "C" {

sp_status sp_build(const sp_circuit_desc *circuit, void *cuda_stream, sp_program **out)
{
    if (!out) return set_error(SP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!circuit) return set_error(SP_ERR_INVALID_ARG, "circuit is NULL");
    sp_program *P = host_alloc_fails() ? nullptr : new (std::nothrow) sp_program();
    if (!P) return set_error(SP_ERR_OOM, "host allocation of the program failed");
    g_live_host++;
    sp_status st = build_program(circuit, (cudaStream_t)cuda_stream, P);
    if (st != SP_OK) {
        cudaStreamSynchronize((cudaStream_t)cuda_stream);
        cudaGetLastError();
        release(P);
        return st;
    }
    *out = P;
    return SP_OK;
}

sp_status sp_save(const sp_program *P, void *buf, size_t cap, size_t *size)
{
    if (!P) return set_error(SP_ERR_INVALID_ARG, "prog is NULL");
    if (!buf && !size) return set_error(SP_ERR_INVALID_ARG, "buf and size are both NULL");
    int cur = -1;
    if (buf) {
        SP_CUDA(cudaGetDevice(&cur));
        if (cur != P->device) SP_CUDA(cudaSetDevice(P->device));
    }
    const sp_status st = save_program(P, buf, cap, size);
    if (buf && cur != P->device) cudaSetDevice(cur);
    return st;
}

sp_status sp_load(const void *buf, size_t size, void *cuda_stream, sp_program **out)
{
    if (!out) return set_error(SP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    SP_TRY(check_saved(buf, size));
    sp_program *P = host_alloc_fails() ? nullptr : new (std::nothrow) sp_program();
    if (!P) return set_error(SP_ERR_OOM, "host allocation of the program failed");
    g_live_host++;
    const auto t0 = std::chrono::steady_clock::now();
    sp_status st = load_program(buf, size, (cudaStream_t)cuda_stream, P);
    if (st != SP_OK) {
        cudaStreamSynchronize((cudaStream_t)cuda_stream);
        cudaGetLastError();
        release(P);
        return st;
    }
    P->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = P;
    return SP_OK;
}

sp_status sp_info(const sp_program *P, sp_info_t *o)
{
    if (!P || !o) return set_error(SP_ERR_INVALID_ARG, "NULL argument");
    memset(o, 0, sizeof *o);
    o->num_qubits = P->n;
    o->num_measurements = (uint64_t)P->n_meas;
    o->num_detectors = (uint64_t)P->n_det;
    o->num_observables = (uint64_t)P->n_obs;
    o->num_symbols = (uint64_t)P->n_sym;
    o->num_channels = (uint64_t)P->n_ch;
    o->num_random = (uint64_t)P->n_rand;
    o->nnz_rows = (uint64_t)P->nnz_rows;
    o->nnz_delta = (uint64_t)P->nnz_delta;
    o->log_words = (uint64_t)P->log_len;
    o->density = P->density;
    o->path = P->path;
    o->fused_tile_shots = 32 * P->fused_tw;
    o->fused_variant = P->fused_tw ? P->fused_unroll : 0;
    o->fused_ctas_per_sm = P->fused_tw ? P->fused_ctas_per_sm : 0;
    o->autotune_launches = P->autotune_launches;
    o->stream = P->stream;
    o->chunk_shots = (uint64_t)P->chunk_shots;
    o->build_ms = P->build_ms;
    for (int k = 0; k < 5; k++) o->path_probe_ms[k] = P->path_probe_ms[k];
    o->live_blocks = (uint64_t)P->n_blk_live;
    return SP_OK;
}

sp_status sp_sample(sp_program *P, uint64_t seed, uint64_t shot0, uint64_t nshots,
                    uint64_t *d_meas, uint64_t *d_det, uint64_t *d_obs, void *cuda_stream)
{
    if (!P) return set_error(SP_ERR_INVALID_ARG, "prog is NULL");
    sp_status st;
    if ((st = check_ptr(d_meas, "d_meas")) || (st = check_ptr(d_det, "d_det")) || (st = check_ptr(d_obs, "d_obs")))
        return st;
    if (nshots == 0) return SP_OK;
    if (shot0 + nshots < shot0) return set_error(SP_ERR_INVALID_ARG, "shot range overflows 64 bits");
    return sample_range(P, seed, shot0, nshots, d_meas, d_det, d_obs, (cudaStream_t)cuda_stream);
}

sp_status sp_sample_host(sp_program *P, uint64_t seed, uint64_t shot0, uint64_t nshots,
                         uint64_t *h_meas, uint64_t *h_det, uint64_t *h_obs, void *cuda_stream)
{
    if (!P) return set_error(SP_ERR_INVALID_ARG, "prog is NULL");
    if (nshots == 0) return SP_OK;
    if (shot0 + nshots < shot0) return set_error(SP_ERR_INVALID_ARG, "shot range overflows 64 bits");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int64_t wm = words64(P->n_meas), wd = words64(P->n_det), wo = words64(P->n_obs);
    const int64_t per_shot = wm + wd + wo;
    // pipeline granularity: at most the sampling chunk, at most 64 MiB of records
    int64_t piece = std::min<int64_t>(P->chunk_shots, std::max<int64_t>(1024, (64 << 20) / std::max<int64_t>(per_shot * 8, 8)));
    piece = std::max<int64_t>(1024, (piece / 1024) * 1024);
    // the copy of the last piece is the one nothing overlaps: keep it short
    // (one wave of the fused kernel's tiles, else 1/8 of a piece)
    int64_t tail = std::max<int64_t>(1024, piece / 8);
    if (P->path == SP_PATH_FUSED && P->fused_tw) {
        // whole waves of the fused kernel's tiles, so that no piece ends in a
        // partly filled wave
        const int64_t wave = (int64_t)P->num_sms * P->fused_ctas_per_sm * 32 * P->fused_tw;
        if (wave > 0 && piece > wave) piece = (piece / wave) * wave;
        if (wave > 0) tail = std::min<int64_t>(piece, wave);
    }
    sp_status st = SP_OK;
    if (uses_staged_scratch(P)) {
        st = ensure_scratch(P, (size_t)std::min<uint64_t>(nshots, (uint64_t)piece));
        if (st != SP_OK) return st;
    }
    const size_t stage_words = (size_t)piece * (size_t)per_shot;
    if (P->d_out_stage_bytes < 2 * stage_words * 8) {
        if (P->d_out_stage) dev_free(P->d_out_stage);
        P->d_out_stage = nullptr;
        P->d_out_stage_bytes = 0;
        if (dev_alloc((void **)&P->d_out_stage, 2 * stage_words * 8) != cudaSuccess) {
            cudaGetLastError();
            P->d_out_stage = nullptr;
            return set_error(SP_ERR_OOM, "cudaMalloc of the output staging buffers failed");
        }
        P->d_out_stage_bytes = 2 * stage_words * 8;
    }
    if (!P->copy_stream) SP_CUDA(cudaStreamCreateWithFlags(&P->copy_stream, cudaStreamNonBlocking));
    for (cudaEvent_t &e : P->ev)
        if (!e) SP_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    // ev[0..1]: chunk i computed in stage i%2; ev[2..3]: stage i%2 copied out
    bool used[2] = {false, false};
    int64_t i = 0;
    for (uint64_t done = 0, n = 0; done < nshots; done += n, i++) {
        const uint64_t left = nshots - done;
        // full pieces; the last one that would exceed 2 tails leaves one tail behind
        n = left > (uint64_t)piece ? (uint64_t)piece : left > 2 * (uint64_t)tail ? left - (uint64_t)tail : left;
        const int b = (int)(i & 1);
        uint64_t *dm = P->d_out_stage + (size_t)b * stage_words;
        uint64_t *dd = dm + (size_t)piece * wm;
        uint64_t *dob = dd + (size_t)piece * wd;
        if (used[b]) SP_CUDA(cudaStreamWaitEvent(s, P->ev[2 + b], 0));
        st = sample_chunk(P, seed, shot0 + done, (uint64_t)n, h_meas ? dm : nullptr, h_det ? dd : nullptr,
                          h_obs ? dob : nullptr, s);
        if (st != SP_OK) return st;
        SP_CUDA(cudaEventRecord(P->ev[b], s));
        SP_CUDA(cudaStreamWaitEvent(P->copy_stream, P->ev[b], 0));
        if (h_meas && wm) SP_CUDA(cudaMemcpyAsync(h_meas + done * wm, dm, (size_t)n * wm * 8, cudaMemcpyDeviceToHost, P->copy_stream));
        if (h_det && wd) SP_CUDA(cudaMemcpyAsync(h_det + done * wd, dd, (size_t)n * wd * 8, cudaMemcpyDeviceToHost, P->copy_stream));
        if (h_obs && wo) SP_CUDA(cudaMemcpyAsync(h_obs + done * wo, dob, (size_t)n * wo * 8, cudaMemcpyDeviceToHost, P->copy_stream));
        SP_CUDA(cudaEventRecord(P->ev[2 + b], P->copy_stream));
        used[b] = true;
    }
    SP_CUDA(cudaStreamSynchronize(P->copy_stream));
    SP_CUDA(cudaStreamSynchronize(s));
    if (P->path == SP_PATH_TENSOR && P->d_tc_status) {
        int32_t v = 0;
        return sp_device_status(P, &v);
    }
    return SP_OK;
}

sp_status sp_sample_batch(sp_program *const *progs, uint32_t nprog, const uint64_t *seeds,
                          const uint64_t *nshots, uint64_t *const *d_meas, uint64_t *const *d_det,
                          uint64_t *const *d_obs, void *cuda_stream)
{
    if (nprog == 0) return SP_OK;
    if (!progs || !seeds || !nshots) return set_error(SP_ERR_INVALID_ARG, "NULL array argument");
    for (uint32_t i = 0; i < nprog; i++) {
        if (!progs[i]) return set_error(SP_ERR_INVALID_ARG, "progs[" + std::to_string(i) + "] is NULL");
    }
    for (uint32_t i = 0; i < nprog; i++) {
        for (uint64_t *const *arr : {d_meas, d_det, d_obs}) {
            if (!arr) continue;
            sp_status st = check_ptr(arr[i], "output");
            if (st != SP_OK) return st;
        }
    }
    return sample_batch(progs, nprog, seeds, nshots, d_meas, d_det, d_obs, (cudaStream_t)cuda_stream);
}

sp_status sp_expect(sp_program *P, const float *d_p, float *d_logE, void *cuda_stream)
{
    if (!P || !d_logE) return set_error(SP_ERR_INVALID_ARG, "NULL argument");
    return expect_fwd(P, d_p, d_logE, (cudaStream_t)cuda_stream);
}

sp_status sp_expect_sign(sp_program *P, const float *d_p, float *d_sign, void *cuda_stream)
{
    if (!P || !d_sign) return set_error(SP_ERR_INVALID_ARG, "NULL argument");
    return expect_sign(P, d_p, d_sign, (cudaStream_t)cuda_stream);
}

sp_status sp_expect_grad(sp_program *P, const float *d_p, const float *d_grad_logE, float *d_grad_p,
                         void *cuda_stream)
{
    if (!P || !d_grad_logE || !d_grad_p) return set_error(SP_ERR_INVALID_ARG, "NULL argument");
    return expect_bwd(P, d_p, d_grad_logE, d_grad_p, (cudaStream_t)cuda_stream);
}

sp_status sp_export_rows(const sp_program *P, int32_t which, uint64_t *h_out, uint64_t row_words)
{
    if (!P || !h_out) return set_error(SP_ERR_INVALID_ARG, "NULL argument");
    if (which < 0 || which > 2) return set_error(SP_ERR_INVALID_ARG, "which must be 0, 1 or 2");
    const int64_t need = words64(P->n_sym + 1);
    if ((int64_t)row_words < need) return set_error(SP_ERR_INVALID_ARG, "row_words too small");
    const int64_t row0 = which == 0 ? 0 : (which == 1 ? P->n_meas : P->n_meas + P->n_det);
    const int64_t cnt = which == 0 ? P->n_meas : (which == 1 ? P->n_det : P->n_obs);
    if (cnt == 0) return SP_OK;
    std::vector<uint32_t> buf((size_t)cnt * P->apitch);
    SP_CUDA(cudaMemcpy(buf.data(), P->d_A + (size_t)row0 * P->apitch, buf.size() * 4, cudaMemcpyDeviceToHost));
    for (int64_t r = 0; r < cnt; r++) {
        uint64_t *dst = h_out + (size_t)r * row_words;
        memset(dst, 0, row_words * 8);
        memcpy(dst, buf.data() + (size_t)r * P->apitch, (size_t)std::min<int64_t>(P->apitch * 4, (int64_t)row_words * 8));
    }
    return SP_OK;
}

sp_status sp_export_channels(const sp_program *P, uint32_t *h_T, uint8_t *h_kind, uint64_t *h_sym0)
{
    if (!P) return set_error(SP_ERR_INVALID_ARG, "prog is NULL");
    if (P->n_ch == 0) return SP_OK;
    if (h_T) SP_CUDA(cudaMemcpy(h_T, P->d_chT, (size_t)P->n_ch * 4, cudaMemcpyDeviceToHost));
    if (h_kind) SP_CUDA(cudaMemcpy(h_kind, P->d_chKind, (size_t)P->n_ch, cudaMemcpyDeviceToHost));
    if (h_sym0) {
        std::vector<uint32_t> s0((size_t)P->n_ch);
        SP_CUDA(cudaMemcpy(s0.data(), P->d_chSym0, (size_t)P->n_ch * 4, cudaMemcpyDeviceToHost));
        for (int64_t c = 0; c < P->n_ch; c++) h_sym0[c] = s0[c];
    }
    return SP_OK;
}

sp_status sp_set_path(sp_program *P, int32_t path)
{
    if (!P) return set_error(SP_ERR_INVALID_ARG, "prog is NULL");
    if (P->stream == 2 && path != SP_PATH_FUSED && !(path == SP_PATH_AUTO && P->build_path == SP_PATH_FUSED))
        return set_error(SP_ERR_INVALID_ARG, "the grouped draw (stream 2) runs on the fused path only");
    if (path == SP_PATH_AUTO) {
        P->path = P->build_path;
        reconfigured(P);
        return SP_OK;
    }
    if (path == SP_PATH_FUSED && !P->fused_tw)
        return set_error(SP_ERR_INVALID_ARG, "the fused path is unavailable for this program");
    if (path == SP_PATH_TENSOR && !tensor_path_available(P))
        return set_error(SP_ERR_INVALID_ARG, "the tensor-core path is unavailable for this program or device");
    if (path != SP_PATH_SPARSE && path != SP_PATH_FUSED && path != SP_PATH_DENSE && path != SP_PATH_TENSOR)
        return set_error(SP_ERR_INVALID_ARG, "unsupported path");
    P->path = path;
    reconfigured(P);
    return SP_OK;
}

sp_status sp_set_fused_config(sp_program *P, int32_t tile_shots, int32_t variant)
{
    if (!P) return set_error(SP_ERR_INVALID_ARG, "prog is NULL");
    if (tile_shots != 32 && tile_shots != 64 && tile_shots != 128)
        return set_error(SP_ERR_INVALID_ARG, "tile_shots must be 32, 64 or 128");
    const sp_status st = fused_select(P, tile_shots / 32, variant);
    if (st == SP_OK) reconfigured(P);
    return st;
}

sp_status sp_set_stream(sp_program *P, int32_t stream)
{
    if (!P) return set_error(SP_ERR_INVALID_ARG, "prog is NULL");
    if (stream != 1 && stream != 2) return set_error(SP_ERR_INVALID_ARG, "stream must be 1 or 2");
    if (stream == 2) {
        if (!P->fused_tw) return set_error(SP_ERR_INVALID_ARG, "the grouped draw (stream 2) needs the fused path");
        const sp_status st = ensure_grouped(P, nullptr);
        if (st != SP_OK) return st;
        P->path = SP_PATH_FUSED;
    }
    const int old = P->stream;
    P->stream = stream;
    reconfigured(P);
    // the launch shape is tuned per stream (cached per circuit shape)
    if (stream != old && P->fused_tw) {
        const sp_status st = autotune(P, nullptr);
        if (st != SP_OK) {
            P->stream = old;
            return st;
        }
    }
    return SP_OK;
}

sp_status sp_device_status(sp_program *P, int32_t *status)
{
    if (!P || !status) return set_error(SP_ERR_INVALID_ARG, "prog and status must not be NULL");
    *status = 0;
    if (!P->d_tc_status) return SP_OK;
    int v = 0;
    SP_CUDA(cudaDeviceSynchronize());
    SP_CUDA(cudaMemcpy(&v, P->d_tc_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (v) SP_CUDA(cudaMemset(P->d_tc_status, 0, sizeof(int)));
    *status = v;
    if (v) return set_error(SP_ERR_TIMEOUT, "a tensor-core tile gave up on a bounded wait; its records were not written");
    return SP_OK;
}

sp_status sp_set_wait_limit(sp_program *P, uint64_t ns)
{
    if (!P) return set_error(SP_ERR_INVALID_ARG, "prog is NULL");
    P->tc_wait_ns = ns;
    return SP_OK;
}

sp_status sp_set_chunk(sp_program *P, uint64_t chunk_shots)
{
    if (!P) return set_error(SP_ERR_INVALID_ARG, "prog is NULL");
    if (chunk_shots % 1024) return set_error(SP_ERR_INVALID_ARG, "chunk_shots must be a multiple of 1024");
    P->chunk_shots = chunk_shots ? (int64_t)chunk_shots : default_chunk(P);
    reconfigured(P);
    return SP_OK;
}

sp_status sp_profile_enable(sp_program *P, int32_t on)
{
    if (!P) return set_error(SP_ERR_INVALID_ARG, "prog is NULL");
    P->profiling = on != 0;
    return SP_OK;
}

sp_status sp_profile_read(sp_program *P, double *ms, uint64_t *launches)
{
    if (!P) return set_error(SP_ERR_INVALID_ARG, "prog is NULL");
    double acc[SP_KERNEL_CLASSES] = {0};
    uint64_t cnt[SP_KERNEL_CLASSES] = {0};
    for (auto &pe : P->ev_pending) {
        SP_CUDA(cudaEventSynchronize(pe.second.second));
        float t = 0.f;
        SP_CUDA(cudaEventElapsedTime(&t, pe.second.first, pe.second.second));
        if (pe.first >= 0 && pe.first < SP_KERNEL_CLASSES) {
            acc[pe.first] += t;
            cnt[pe.first] += 1;
        }
        P->ev_pool.push_back(pe.second.first);
        P->ev_pool.push_back(pe.second.second);
    }
    P->ev_pending.clear();
    for (int k = 0; k < SP_KERNEL_CLASSES; k++) {
        if (ms) ms[k] = acc[k];
        if (launches) launches[k] = cnt[k];
    }
    return SP_OK;
}

sp_status sp_debug_fail_alloc(int64_t after)
{
    g_fail_after.store(after < 0 ? -1 : after);
    return SP_OK;
}

sp_status sp_debug_live_allocs(int64_t *device_allocs, int64_t *host_programs)
{
    if (device_allocs) *device_allocs = g_live_dev.load();
    if (host_programs) *host_programs = g_live_host.load();
    return SP_OK;
}

sp_status sp_batch_plans(uint32_t *count, uint32_t *capacity)
{
    if (count) *count = (uint32_t)batch_plan_count();
    if (capacity) *capacity = (uint32_t)BATCH_MAX_PLANS;
    return SP_OK;
}

void sp_free(sp_program *P) { release(P); }

const char *sp_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
