// Saving and restoring a built program (sp_save / sp_load).
//
// What Algorithm 1's initialization produces is the coefficient rows of
// every measurement, detector and observable over the symbols (Eq. sampling:
// m_j = c_j XOR <a_j, s>) together with the channel of each symbol and its
// distribution (Sec. 3.1).  Everything else the library holds is derived
// from those and from the device (sampler tables, expectation incidence,
// fused-kernel program, launch shapes), so a saved program carries only:
//   - the channel table (threshold, kind, probability, first symbol) and the
//     probability of each non-random channel in double precision;
//   - the detector and observable definitions (XORs of measurement rows);
//   - the rows in the parent-delta form the sampler runs on: row j is its
//     parent's row (an earlier row, at most PARENT_LOOKBACK back, or none)
//     XOR its own symbols, and its constant bit.
// sp_load checks every field on the host before it touches the device,
// rebuilds the rows on the device (k_scatter_own, k_fold_parents), and then
// runs the same finishing steps as sp_build.  The traversal (the part of
// sp_build whose cost grows with circuit depth) is not repeated.
//
// Layout: a SaveHeader, then the payload sections in the order of
// section_sizes(), each starting at a multiple of 8 bytes.  All integers
// and floats are little-endian (the writer's byte order is recorded and
// must match the reader's).
#include <algorithm>
#include <cstring>
#include <vector>

#include "sp_internal.h"

namespace sp {
namespace {

constexpr char SAVE_MAGIC[8] = {'S', 'Y', 'M', 'P', 'H', 'A', 'S', 'E'};
constexpr uint32_t SAVE_VERSION = 1;
constexpr uint32_t SAVE_ENDIAN = 0x01020304u;

struct SaveHeader {
    char magic[8];
    uint32_t version;
    uint32_t endian;                 // SAVE_ENDIAN as stored by the writer
    uint32_t header_bytes;           // sizeof(SaveHeader)
    uint32_t max_parent_distance;    // PARENT_LOOKBACK of the writer
    uint64_t n, n_meas, n_det, n_obs, n_sym, n_ch, log_len, nnz_rows, nnz_delta;
    uint64_t n_fault, n_xrefs;
    uint64_t payload_bytes;
    uint64_t checksum;               // FNV-1a (64-bit) of the payload
};
static_assert(sizeof(SaveHeader) == 128, "SaveHeader layout");

enum Section { S_CHT, S_CHKIND, S_CHP, S_CHSYM0, S_FAULTP, S_XOFF, S_XREFS, S_PARENT, S_CONST, S_ROWOFF, S_IDX, S_COUNT };

uint64_t pad8(uint64_t x) { return (x + 7) & ~7ull; }

// bytes of each payload section, from the header's counts
void section_sizes(const SaveHeader &h, uint64_t sz[S_COUNT])
{
    const uint64_t R = h.n_meas + h.n_det + h.n_obs;
    sz[S_CHT] = 4 * h.n_ch;
    sz[S_CHKIND] = h.n_ch;
    sz[S_CHP] = 4 * h.n_ch;
    sz[S_CHSYM0] = 4 * h.n_ch;
    sz[S_FAULTP] = 8 * h.n_fault;
    sz[S_XOFF] = 4 * (h.n_det + h.n_obs + 1);
    sz[S_XREFS] = 4 * h.n_xrefs;
    sz[S_PARENT] = 4 * R;
    sz[S_CONST] = R;
    sz[S_ROWOFF] = 4 * (R + 1);
    sz[S_IDX] = 4 * h.nnz_delta;
}

uint64_t fnv1a(const uint8_t *p, uint64_t n)
{
    uint64_t x = 0xcbf29ce484222325ull;
    for (uint64_t i = 0; i < n; i++) {
        x ^= p[i];
        x *= 0x100000001b3ull;
    }
    return x;
}

sp_status bad(const std::string &what) { return set_error(SP_ERR_INVALID_ARG, "saved program: " + what); }

// A parsed blob: pointers into the caller's buffer (no copies).
struct Parsed {
    SaveHeader h;
    const uint8_t *sec[S_COUNT];
    uint64_t R = 0;
};

int kind_width(uint8_t k) { return k == CK_DEP2 ? 4 : k == CK_DEP1 ? 2 : 1; }

// Every check sp_load makes before it allocates anything.
sp_status parse(const void *buf, size_t size, Parsed &P)
{
    if (!buf) return set_error(SP_ERR_INVALID_ARG, "buf is NULL");
    if (size < sizeof(SaveHeader)) return bad("shorter than its header");
    memcpy(&P.h, buf, sizeof(SaveHeader));
    const SaveHeader &h = P.h;
    if (memcmp(h.magic, SAVE_MAGIC, 8) != 0) return bad("not a SymPhase program (magic)");
    if (h.endian != SAVE_ENDIAN) return bad("written with another byte order");
    if (h.version != SAVE_VERSION) return bad("format version " + std::to_string(h.version) + " (this library reads 1)");
    if (h.header_bytes != sizeof(SaveHeader)) return bad("header size");
    if (h.max_parent_distance != (uint32_t)PARENT_LOOKBACK) return bad("parent distance bound differs");
    if (h.n > 1024) return bad("more than 1024 qubits");
    // bounds that keep every later size computation far from overflow
    const uint64_t LIM = 1ull << 31;
    if (h.n_meas >= LIM || h.n_det >= LIM || h.n_obs >= LIM || h.n_sym >= LIM || h.n_ch >= LIM ||
        h.n_fault >= LIM || h.n_xrefs >= LIM || h.nnz_delta >= (1ull << 32) || h.nnz_rows >= (1ull << 40))
        return bad("a count is out of range");
    P.R = h.n_meas + h.n_det + h.n_obs;
    if (P.R >= LIM) return bad("too many rows");
    uint64_t sz[S_COUNT], total = 0;
    section_sizes(h, sz);
    for (int s = 0; s < S_COUNT; s++) total += pad8(sz[s]);
    if (h.payload_bytes != total) return bad("payload size does not match the counts");
    if ((uint64_t)size != sizeof(SaveHeader) + total) return bad("buffer size does not match the header");
    const uint8_t *pay = static_cast<const uint8_t *>(buf) + sizeof(SaveHeader);
    if (fnv1a(pay, total) != h.checksum) return bad("checksum mismatch");
    uint64_t off = 0;
    for (int s = 0; s < S_COUNT; s++) {
        P.sec[s] = pay + off;
        off += pad8(sz[s]);
    }
    // channel table: the channels cover symbols 1..n_sym in order
    std::vector<uint32_t> T(h.n_ch), s0(h.n_ch);
    std::vector<float> cp(h.n_ch);
    memcpy(T.data(), P.sec[S_CHT], sz[S_CHT]);
    memcpy(s0.data(), P.sec[S_CHSYM0], sz[S_CHSYM0]);
    memcpy(cp.data(), P.sec[S_CHP], sz[S_CHP]);
    const uint8_t *kind = P.sec[S_CHKIND];
    std::vector<double> fp(h.n_fault);
    memcpy(fp.data(), P.sec[S_FAULTP], sz[S_FAULTP]);
    uint64_t next = 1, fault = 0;
    for (uint64_t c = 0; c < h.n_ch; c++) {
        if (kind[c] > CK_RANDOM) return bad("channel " + std::to_string(c) + ": unknown kind");
        if (s0[c] != next) return bad("channel " + std::to_string(c) + ": symbols out of order");
        next += (uint64_t)kind_width(kind[c]);
        if (kind[c] == CK_RANDOM) {
            if (T[c] != 0x80000000u || cp[c] != 0.5f) return bad("channel " + std::to_string(c) + ": random outcome table");
        } else {
            if (fault >= h.n_fault) return bad("fewer probabilities than noise channels");
            const double p = fp[fault++];
            if (!(p >= 0.0 && p <= 1.0)) return bad("channel " + std::to_string(c) + ": probability outside [0, 1]");
            if (T[c] != threshold_of(p) || cp[c] != (float)p)
                return bad("channel " + std::to_string(c) + ": threshold does not match its probability");
        }
    }
    if (fault != h.n_fault) return bad("more probabilities than noise channels");
    if (next != h.n_sym + 1) return bad("the channels do not cover the symbols");
    // detector and observable definitions
    std::vector<uint32_t> xoff(h.n_det + h.n_obs + 1), xrefs(h.n_xrefs);
    memcpy(xoff.data(), P.sec[S_XOFF], sz[S_XOFF]);
    memcpy(xrefs.data(), P.sec[S_XREFS], sz[S_XREFS]);
    if (xoff[0] != 0 || xoff.back() != h.n_xrefs) return bad("detector offsets");
    for (size_t t = 0; t + 1 < xoff.size(); t++)
        if (xoff[t] > xoff[t + 1]) return bad("detector offsets decrease");
    for (uint32_t r : xrefs)
        if (r >= h.n_meas) return bad("a detector refers to a missing measurement");
    // rows: parents, constants, own symbols
    std::vector<int32_t> par(P.R);
    std::vector<uint32_t> roff(P.R + 1);
    memcpy(par.data(), P.sec[S_PARENT], sz[S_PARENT]);
    memcpy(roff.data(), P.sec[S_ROWOFF], sz[S_ROWOFF]);
    const uint8_t *cst = P.sec[S_CONST];
    for (uint64_t j = 0; j < P.R; j++) {
        const int64_t p = par[j];
        if (p != -1 && (p < 0 || p >= (int64_t)j || (int64_t)j - p > PARENT_LOOKBACK))
            return bad("row " + std::to_string(j) + ": parent out of range");
        if (cst[j] > 1) return bad("row " + std::to_string(j) + ": constant bit");
    }
    if (roff[0] != 0 || roff[P.R] != h.nnz_delta) return bad("row offsets");
    std::vector<uint32_t> idx(h.nnz_delta);
    memcpy(idx.data(), P.sec[S_IDX], sz[S_IDX]);
    for (uint64_t j = 0; j < P.R; j++) {
        if (roff[j] > roff[j + 1]) return bad("row offsets decrease");
        for (uint32_t k = roff[j]; k < roff[j + 1]; k++) {
            // symbol - 1, strictly increasing within a row
            if (idx[k] >= h.n_sym) return bad("row " + std::to_string(j) + ": symbol out of range");
            if (k > roff[j] && idx[k] <= idx[k - 1]) return bad("row " + std::to_string(j) + ": symbols not increasing");
        }
    }
    return SP_OK;
}

// Set the bits of row j's own symbols (one warp per row; a row's symbols
// are distinct, so OR is the XOR of the delta form).
__global__ void k_scatter_own(const uint32_t *__restrict__ rowOff, const uint32_t *__restrict__ idx, int64_t nrows,
                              uint32_t *A, int64_t apitch)
{
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (j >= nrows) return;
    const int lane = threadIdx.x & 31;
    for (uint32_t k = rowOff[j] + (uint32_t)lane; k < rowOff[j + 1]; k += 32) {
        const uint32_t s = idx[k] + 1u;
        atomicOr(&A[(size_t)j * apitch + (s >> 5)], 1u << (s & 31));
    }
}

// Fold the parents in: row j := own(j) XOR row(parent j), in row order, and
// its bit 0 := the constant.  Thread = one word column of every row; the
// last PARENT_LOOKBACK finished words of its column wait in shared memory,
// where the parent's word is read.  Eight rows' own words are loaded ahead.
constexpr int FOLD_THREADS = 32;
constexpr int FOLD_AHEAD = 8;

__global__ void __launch_bounds__(FOLD_THREADS) k_fold_parents(uint32_t *A, int64_t apitch, int64_t nrows,
                                                               const int32_t *__restrict__ parent,
                                                               const uint8_t *__restrict__ cst)
{
    extern __shared__ uint32_t ring[];   // [PARENT_LOOKBACK][FOLD_THREADS]
    const int64_t w = (int64_t)blockIdx.x * FOLD_THREADS + threadIdx.x;
    if (w >= apitch) return;
    uint32_t *slot = ring + threadIdx.x;
    for (int64_t j0 = 0; j0 < nrows; j0 += FOLD_AHEAD) {
        uint32_t v[FOLD_AHEAD];
        int32_t pa[FOLD_AHEAD];
#pragma unroll
        for (int i = 0; i < FOLD_AHEAD; i++) {
            const bool in = j0 + i < nrows;
            v[i] = in ? A[(size_t)(j0 + i) * apitch + w] : 0u;
            pa[i] = in ? parent[j0 + i] : -1;
        }
#pragma unroll
        for (int i = 0; i < FOLD_AHEAD; i++) {
            const int64_t j = j0 + i;
            if (j >= nrows) break;
            uint32_t x = v[i];
            if (pa[i] >= 0) x ^= slot[(size_t)(pa[i] % PARENT_LOOKBACK) * FOLD_THREADS];
            if (w == 0) x = (x & ~1u) | cst[j];
            slot[(size_t)(j % PARENT_LOOKBACK) * FOLD_THREADS] = x;
            A[(size_t)j * apitch + w] = x;
        }
    }
}

sp_status alloc_bytes(void **d, size_t bytes)
{
    if (dev_alloc(d, bytes) != cudaSuccess) {
        cudaGetLastError();
        *d = nullptr;
        return set_error(SP_ERR_OOM, "cudaMalloc of a restored program table failed");
    }
    return SP_OK;
}

// count entries from the host, plus one zero entry after them; a buffer
// that was allocated is recorded in *owned (if given) before the copies
template <typename T>
sp_status upload(T **d, const void *src, uint64_t count, cudaStream_t stream, std::vector<void *> *owned = nullptr)
{
    SP_TRY(alloc_bytes(reinterpret_cast<void **>(d), (size_t)(count + 1) * sizeof(T)));
    if (owned) owned->push_back(*d);
    if (count) SP_CUDA(cudaMemcpyAsync(*d, src, (size_t)count * sizeof(T), cudaMemcpyHostToDevice, stream));
    SP_CUDA(cudaMemsetAsync(*d + count, 0, sizeof(T), stream));
    return SP_OK;
}

template <typename T> sp_status download(std::vector<uint8_t> &out, uint64_t at, const T *d, uint64_t count)
{
    if (count) SP_CUDA(cudaMemcpy(out.data() + at, d, (size_t)count * sizeof(T), cudaMemcpyDeviceToHost));
    return SP_OK;
}

}  // namespace

sp_status save_program(const sp_program *P, void *buf, size_t cap, size_t *size)
{
    SaveHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, SAVE_MAGIC, 8);
    h.version = SAVE_VERSION;
    h.endian = SAVE_ENDIAN;
    h.header_bytes = sizeof(SaveHeader);
    h.max_parent_distance = PARENT_LOOKBACK;
    h.n = P->n;
    h.n_meas = (uint64_t)P->n_meas;
    h.n_det = (uint64_t)P->n_det;
    h.n_obs = (uint64_t)P->n_obs;
    h.n_sym = (uint64_t)P->n_sym;
    h.n_ch = (uint64_t)P->n_ch;
    h.log_len = (uint64_t)P->log_len;
    h.nnz_rows = (uint64_t)P->nnz_rows;
    h.nnz_delta = (uint64_t)P->nnz_delta;
    h.n_fault = P->h_fault_p.size();
    h.n_xrefs = P->h_xrefs.size();
    uint64_t sz[S_COUNT], total = 0, off[S_COUNT];
    section_sizes(h, sz);
    for (int s = 0; s < S_COUNT; s++) {
        off[s] = total;
        total += pad8(sz[s]);
    }
    h.payload_bytes = total;
    const size_t need = sizeof(SaveHeader) + (size_t)total;
    if (size) *size = need;
    if (!buf) return SP_OK;
    if (cap < need) return set_error(SP_ERR_INVALID_ARG, "buffer holds " + std::to_string(cap) + " bytes, the program needs " + std::to_string(need));
    if (P->h_xoff.size() != h.n_det + h.n_obs + 1) return set_error(SP_ERR_INVALID_ARG, "program has no detector table");
    std::vector<uint8_t> pay((size_t)total, 0);
    const uint64_t R = h.n_meas + h.n_det + h.n_obs;
    SP_TRY(download(pay, off[S_CHT], P->d_chT, h.n_ch));
    SP_TRY(download(pay, off[S_CHKIND], P->d_chKind, h.n_ch));
    SP_TRY(download(pay, off[S_CHP], P->d_chP, h.n_ch));
    SP_TRY(download(pay, off[S_CHSYM0], P->d_chSym0, h.n_ch));
    if (h.n_fault) memcpy(pay.data() + off[S_FAULTP], P->h_fault_p.data(), sz[S_FAULTP]);
    memcpy(pay.data() + off[S_XOFF], P->h_xoff.data(), sz[S_XOFF]);
    if (h.n_xrefs) memcpy(pay.data() + off[S_XREFS], P->h_xrefs.data(), sz[S_XREFS]);
    SP_TRY(download(pay, off[S_PARENT], P->d_parent, R));
    SP_TRY(download(pay, off[S_CONST], P->d_const, R));
    SP_TRY(download(pay, off[S_ROWOFF], P->d_rowOff, R + 1));
    SP_TRY(download(pay, off[S_IDX], P->d_idx, h.nnz_delta));
    h.checksum = fnv1a(pay.data(), total);
    memcpy(buf, &h, sizeof h);
    if (total) memcpy(static_cast<uint8_t *>(buf) + sizeof h, pay.data(), (size_t)total);
    return SP_OK;
}

sp_status check_saved(const void *buf, size_t size)
{
    Parsed Q;
    return parse(buf, size, Q);
}

sp_status load_program(const void *buf, size_t size, cudaStream_t stream, sp_program *P)
{
    Parsed Q;
    SP_TRY(parse(buf, size, Q));
    const SaveHeader &h = Q.h;
    SP_CUDA(cudaGetDevice(&P->device));
    P->n = (uint32_t)h.n;
    P->n_meas = (int64_t)h.n_meas;
    P->n_det = (int64_t)h.n_det;
    P->n_obs = (int64_t)h.n_obs;
    P->n_rows = (int64_t)Q.R;
    P->n_sym = (int64_t)h.n_sym;
    P->n_ch = (int64_t)h.n_ch;
    P->log_len = (int64_t)h.log_len;
    // the caller's buffer need not be aligned: copy bytes
    P->h_fault_p.resize(h.n_fault);
    P->h_xoff.resize(h.n_det + h.n_obs + 1);
    P->h_xrefs.resize(h.n_xrefs);
    memcpy(P->h_fault_p.data(), Q.sec[S_FAULTP], h.n_fault * 8);
    memcpy(P->h_xoff.data(), Q.sec[S_XOFF], P->h_xoff.size() * 4);
    if (h.n_xrefs) memcpy(P->h_xrefs.data(), Q.sec[S_XREFS], h.n_xrefs * 4);
    // channel table
    SP_TRY(upload(&P->d_chT, Q.sec[S_CHT], h.n_ch, stream));
    SP_TRY(upload(&P->d_chKind, Q.sec[S_CHKIND], h.n_ch, stream));
    SP_TRY(upload(&P->d_chP, Q.sec[S_CHP], h.n_ch, stream));
    SP_TRY(upload(&P->d_chSym0, Q.sec[S_CHSYM0], h.n_ch, stream));
    // coefficient rows from the parent-delta form
    P->apitch = ceil_div(P->n_sym + 1, 32);
    P->apitch = ceil_div(P->apitch, 4) * 4;
    const size_t arows = (size_t)std::max<int64_t>(P->n_rows, 1);
    SP_TRY(alloc_bytes(reinterpret_cast<void **>(&P->d_A), arows * P->apitch * 4));
    SP_CUDA(cudaMemsetAsync(P->d_A, 0, arows * P->apitch * 4, stream));
    struct Tmp {
        std::vector<void *> p;
        ~Tmp() { for (void *x : p) dev_free(x); }
    } tmp;
    uint32_t *d_roff = nullptr, *d_idx = nullptr;
    int32_t *d_par = nullptr;
    uint8_t *d_cst = nullptr;
    SP_TRY(upload(&d_roff, Q.sec[S_ROWOFF], Q.R + 1, stream, &tmp.p));
    SP_TRY(upload(&d_idx, Q.sec[S_IDX], h.nnz_delta, stream, &tmp.p));
    SP_TRY(upload(&d_par, Q.sec[S_PARENT], Q.R, stream, &tmp.p));
    SP_TRY(upload(&d_cst, Q.sec[S_CONST], Q.R, stream, &tmp.p));
    if (Q.R > 0) {
        k_scatter_own<<<(unsigned)ceil_div((int64_t)Q.R, 8), 256, 0, stream>>>(d_roff, d_idx, (int64_t)Q.R, P->d_A,
                                                                                P->apitch);
        const size_t ring = (size_t)PARENT_LOOKBACK * FOLD_THREADS * 4;
        SP_CUDA(cudaFuncSetAttribute(k_fold_parents, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring));
        k_fold_parents<<<(unsigned)ceil_div(P->apitch, FOLD_THREADS), FOLD_THREADS, ring, stream>>>(
            P->d_A, P->apitch, (int64_t)Q.R, d_par, d_cst);
        SP_CUDA(cudaGetLastError());
    }
    SP_TRY(finish_program(P, stream));
    // the rebuilt sampler program must be the one that was saved
    if ((uint64_t)P->nnz_delta != h.nnz_delta || (uint64_t)P->nnz_rows != h.nnz_rows)
        return bad("the rebuilt rows differ from the saved sampler program");
    std::vector<int32_t> par((size_t)Q.R);
    if (Q.R) SP_CUDA(cudaMemcpy(par.data(), P->d_parent, (size_t)Q.R * 4, cudaMemcpyDeviceToHost));
    if (Q.R && memcmp(par.data(), Q.sec[S_PARENT], (size_t)Q.R * 4) != 0)
        return bad("the rebuilt rows choose other parents than the saved program");
    return SP_OK;
}

}  // namespace sp
