/*
 * symphase.h -- C ABI of the GB300 symbolic-phase stabilizer sampler.
 *
 * Method: arXiv 2311.03906 ("Phase symbolization for fast simulation of
 * stabilizer circuits").  One forward pass of the stabilizer tableau with
 * symbolic phases (Sec. 3.2, Eq. stabilizer3, rules Init-C / Init-P /
 * Init-M) turns every measurement into an affine GF(2) form
 *     m_j = c_j XOR <a_j, s>
 * over the fault symbols and the random-measurement symbols (Sec. 3.2.1).
 * Sampling (Sec. 3.2.3, Eq. sampling, Algorithm 1 "Sampling") draws every
 * symbol from its noise channel and evaluates all forms as one GF(2)
 * matrix product.  Detectors and observables are XORs of measurement
 * records; their forms are XORs of the measurement forms.
 *
 * Conventions shared by every entry point
 *   - All functions return an sp_status.  Arguments are validated before
 *     any GPU work is enqueued; on error nothing is launched, the status is
 *     returned and sp_last_error() (thread-local) describes the problem.
 *     No function aborts the process.
 *   - Pointers named d_* are caller-owned DEVICE memory; h_* are caller-
 *     owned HOST memory.  The library never frees caller memory.
 *   - cuda_stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  sp_sample / sp_expect / sp_expect_grad / sp_sample_batch only
 *     enqueue work on it and return without synchronising.
 *   - Records are bit-packed, shot-major, little-endian: record r of shot t
 *     is bit (r mod 64) of word t*ceil(n/64) + r/64 of a uint64_t array.
 *     Pad bits of the last word of every shot are written as zero.
 *   - Symbols are numbered in op order starting at 1 (symbol 0 is the
 *     constant): a noise channel's symbols when the op is reached
 *     (X/Y/Z_ERROR: 1; DEPOLARIZE1: 2 = x,z; DEPOLARIZE2: 4 = x_a,z_a,x_b,z_b),
 *     a random measurement's symbol when it happens (Sec. 3.1: "symbols
 *     induced by random measurements").  Channels are numbered the same way.
 *   - Draws: Philox4x32-10, key (seed lo32, seed hi32), counter (shot lo32,
 *     shot hi32, channel/4, 0), word channel%4 = u.  A channel fires when
 *     u < T, T = floor(p*2^32) (p = 1 gives 2^32-1); a random-measurement
 *     channel has T = 2^31.  DEPOLARIZE1/2 then take k = floor(u*m/T)
 *     (m = 3 / 15) and symbol s0+i gets bit i of k+1.  Records depend only on
 *     (seed, global shot index), so any chunking of a shot range gives the
 *     same bits.
 */
#ifndef SYMPHASE_H
#define SYMPHASE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SP_API __attribute__((visibility("default")))
#else
#define SP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SP_OK = 0,
    SP_ERR_INVALID_ARG = 1,              /* bad pointer, size, target, probability, look-back */
    SP_ERR_UNSUPPORTED_OP = 2,           /* unknown opcode */
    SP_ERR_NONDETERMINISTIC_DETECTOR = 3,/* a detector/observable depends on a random outcome */
    SP_ERR_OOM = 4,                      /* device or host allocation failed */
    SP_ERR_CUDA = 5,                     /* a CUDA runtime call failed */
    SP_ERR_TIMEOUT = 6,                  /* a device-side bounded wait gave up */
    SP_ERR_TOO_LARGE = 7                 /* circuit beyond the supported size (qubits > 1024) */
} sp_status;

/* Op codes of sp_op.opcode (the circuit grammar). */
enum {
    SP_OP_H = 0, SP_OP_S = 1, SP_OP_CX = 2,           /* Clifford gates (Init-C) */
    SP_OP_X = 3, SP_OP_Y = 4, SP_OP_Z = 5,            /* Pauli gates (Fact 1) */
    SP_OP_M = 6, SP_OP_MR = 7, SP_OP_R = 8,           /* Z measurement, measure+reset, reset (Init-M) */
    SP_OP_X_ERROR = 9, SP_OP_Y_ERROR = 10, SP_OP_Z_ERROR = 11,
    SP_OP_DEPOLARIZE1 = 12, SP_OP_DEPOLARIZE2 = 13,   /* Pauli faults (Init-P, Sec. 3.1 channels) */
    SP_OP_DETECTOR = 14, SP_OP_OBSERVABLE_INCLUDE = 15,
    SP_OP_TICK = 16,
    SP_OP_X_IF = 17, SP_OP_Y_IF = 18, SP_OP_Z_IF = 19  /* feed-forward: conditional Paulis (Sec. 6) */
};

/* One op.  Gate / noise / measurement ops apply to each target in turn
 * (CX and DEPOLARIZE2 to consecutive pairs).  DETECTOR and
 * OBSERVABLE_INCLUDE targets are look-backs k >= 1 meaning rec[-k].
 * X_IF / Y_IF / Z_IF targets are pairs (k, q): the Pauli on qubit q is
 * applied when record rec[-k] is 1, i.e. the conditional Pauli P^e with e
 * that record's affine form (the conditional Paulis of Sec. 6, of which a
 * reset's X^e is the special case on the measured qubit).
 * arg: probability for noise ops, observable index for
 * OBSERVABLE_INCLUDE, ignored otherwise. */
typedef struct {
    uint32_t opcode;
    uint32_t ntargets;
    const uint32_t *targets;
    double arg;
} sp_op;

typedef struct {
    uint32_t num_qubits;   /* <= 1024 */
    uint32_t num_ops;
    const sp_op *ops;
} sp_circuit_desc;

/* Sampler variants for the GF(2) product. */
enum {
    SP_PATH_AUTO = 0,      /* chosen at build time from the measured density */
    SP_PATH_SPARSE = 1,    /* symbol-index XOR gather over bit-sliced shots */
    SP_PATH_DENSE = 2,     /* AND/XOR over shot-major words, then popcount parity (CUDA cores) */
    SP_PATH_FUSED = 3,     /* draw + sparse product + epilogue in one kernel, tile in shared memory */
    SP_PATH_TENSOR = 4     /* 0/1 FP8 tensor-core contraction (tcgen05), exact FP32 sums, parity */
};

typedef struct {
    uint64_t num_qubits;
    uint64_t num_measurements;     /* recorded (M, MR) */
    uint64_t num_detectors;
    uint64_t num_observables;
    uint64_t num_symbols;          /* n_s (excluding the constant) */
    uint64_t num_channels;         /* fault channels + random-measurement channels */
    uint64_t num_random;           /* random-measurement symbols */
    uint64_t nnz_rows;             /* nonzero symbol coefficients over all record rows */
    uint64_t nnz_delta;            /* after parent-delta encoding */
    uint64_t log_words;            /* length of the traversal's row-operation log */
    double density;                /* nnz_rows / (rows * n_s) */
    int32_t path;                  /* SP_PATH_SPARSE, SP_PATH_DENSE, SP_PATH_FUSED or SP_PATH_TENSOR */
    int32_t fused_tile_shots;      /* shots per fused tile (32, 64 or 128; 0 = fused path unavailable) */
    int32_t fused_variant;         /* 1, or 2 = the 64/128-shot kernel built for one CTA per SM */
    int32_t fused_ctas_per_sm;     /* resident CTAs per SM of the chosen fused kernel */
    int32_t autotune_launches;     /* fused-kernel launches the build-time autotuner made */
    int32_t stream;                /* fault-draw stream: 1 per-channel Philox (default), 2 grouped (sp_set_stream) */
    uint64_t chunk_shots;          /* shots per internal sampling chunk */
    double build_ms;               /* wall time of sp_build */
    double path_probe_ms[5];       /* build-time probe of 32,768 shots per SP_PATH_* (0 = not timed: the
                                      dense forms are timed only where >= 1 % of the coefficients are set) */
    uint64_t live_blocks;          /* 4-channel blocks the per-channel draw evaluates per shot: those with a
                                      channel that can fire and whose symbols some measurement row holds
                                      (the others change no record and are skipped) */
} sp_info_t;

typedef struct sp_program sp_program;   /* opaque, library-owned */

/*
 * sp_build -- Algorithm 1 "Initialization": traverse the circuit once with
 * symbolic phases (Init-C, Init-P, Init-M of Sec. 3.2.2) on the GPU and keep
 * the coefficient rows of every measurement, detector and observable plus
 * the sampler program on the current device.
 *   circuit      host description; read only during the call.
 *   cuda_stream  stream for the build kernels; sp_build synchronises it.
 *   out          receives a program to release with sp_free.
 * Errors: INVALID_ARG (target >= num_qubits, CX on one qubit, p outside
 * [0,1], look-back beyond the records so far), UNSUPPORTED_OP,
 * TOO_LARGE (num_qubits > 1024), NONDETERMINISTIC_DETECTOR, OOM, CUDA.
 */
SP_API sp_status sp_build(const sp_circuit_desc *circuit, void *cuda_stream, sp_program **out);

/* sp_info -- sizes and statistics of a built program (host only). */
SP_API sp_status sp_info(const sp_program *prog, sp_info_t *out);

/*
 * sp_save -- write a built program to a host buffer, so that sp_load can
 * restore it without repeating the traversal of Algorithm 1
 * "Initialization".  The blob holds what that traversal produces: the
 * channel table (Sec. 3.1 distributions: threshold, kind, probability and
 * first symbol of each channel), the detector and observable definitions,
 * and the coefficient rows of Eq. sampling in the sampler's parent-delta
 * form (each row = an earlier row XOR its own symbols, plus its constant).
 * Format: a 128-byte header (magic "SYMPHASE", version 1, byte-order mark,
 * counts, payload size, FNV-1a-64 checksum of the payload), then the
 * sections, each 8-byte aligned; little-endian.
 *   buf   host buffer of cap bytes, or NULL to ask for the size only.
 *   size  receives the blob's size in bytes (may be NULL when buf is set).
 * Synchronous (copies the tables back from the program's device); the
 * program is unchanged.  Errors: INVALID_ARG (NULL prog, buf and size both
 * NULL, cap smaller than the blob), CUDA.
 */
SP_API sp_status sp_save(const sp_program *prog, void *buf, size_t cap, size_t *size);

/*
 * sp_load -- rebuild a program written by sp_save on the current device.
 * Every field of the blob is checked on the host before any device call:
 * magic, version, byte order, counts against the buffer size, checksum,
 * the channel table (symbols 1..n in order, each threshold equal to
 * floor(p * 2^32) of its probability, random outcomes at 1/2), detector
 * references, parent distances (<= 512 rows back), symbol ranges and
 * order.  Then the coefficient rows are rebuilt on the device and the
 * sampler program, expectation tables, fused-kernel program and launch
 * shapes are derived from them as sp_build does; the rebuilt sampler
 * program is compared with the saved one.  Records sampled from the loaded
 * program equal those of the saved program for every seed and shot.
 *   buf, size    the blob (read only during the call).
 *   cuda_stream  stream for the rebuild; sp_load synchronises it.
 *   out          receives a program to release with sp_free.
 * Errors: INVALID_ARG (a malformed or inconsistent blob), OOM, CUDA.
 */
SP_API sp_status sp_load(const void *buf, size_t size, void *cuda_stream, sp_program **out);

/*
 * sp_sample -- Algorithm 1 "Sampling" (Eq. sampling) for shots
 * shot0 .. shot0+nshots-1: draw every symbol (Sec. 3.1 distributions,
 * Philox keyed by (seed, shot, channel)), then evaluate all forms.
 *   d_meas  nshots * ceil(num_measurements/64) uint64 words, or NULL to skip
 *   d_det   nshots * ceil(num_detectors/64) words, or NULL
 *   d_obs   nshots * ceil(num_observables/64) words, or NULL
 * Internal scratch (fault-bit and record tiles) is owned by the program and
 * reused, so calls on one program must not overlap on different streams.
 * Errors: INVALID_ARG (NULL prog, misaligned pointer), OOM, CUDA.
 */
SP_API sp_status sp_sample(sp_program *prog, uint64_t seed, uint64_t shot0, uint64_t nshots,
                    uint64_t *d_meas, uint64_t *d_det, uint64_t *d_obs, void *cuda_stream);

/*
 * sp_sample_host -- the same records written to HOST buffers (layout as in
 * sp_sample).  Shots are produced in chunks on the device and copied back
 * while the next chunk is computed; pinned host memory gives full speed.
 * Synchronises the stream before returning.
 */
SP_API sp_status sp_sample_host(sp_program *prog, uint64_t seed, uint64_t shot0, uint64_t nshots,
                         uint64_t *h_meas, uint64_t *h_det, uint64_t *h_obs, void *cuda_stream);

/*
 * sp_sample_static -- the records of sp_sample (same arguments, layout and
 * bits) computed without allocating any memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- a process whose GPU memory is already reserved in full by
 * another allocator (a caching allocator or a pool that owns the device),
 * a latency-critical path that cannot accept an allocation's implicit
 * device synchronisation, or a host application that forbids its plugins to
 * allocate device memory.
 *   Scratch: one fixed 32 MiB device array, reserved on every GPU that
 *   loads the library and held until the process exits.  Shots are
 *   processed in chunks of as many 32-shot words as fit:
 *   32 * floor(8 Mi / (num_symbols + num_rows)) shots per chunk.
 *   Limit: a program with num_symbols + num_rows > 8,388,608 (more than
 *   32 MiB per 32 shots) is rejected with SP_ERR_TOO_LARGE.
 *   Set-up: the first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress, with that device current) and caches it for the
 *   life of the process, so the device's primary context must not be reset
 *   (cudaDeviceReset) after it; make that first call before any stream
 *   capture on the device.  The program must live on the current device.
 *   Sharing: every call on a device uses the same array and leaves its last
 *   contents there.  Calls whose work overlaps on the GPU (different
 *   streams, or different host threads) race on it and must be ordered by
 *   the caller; calls on one stream are ordered by the stream.
 * Errors: INVALID_ARG (NULL prog, misaligned pointer, program of another
 * device), TOO_LARGE, CUDA.
 */
SP_API sp_status sp_sample_static(sp_program *prog, uint64_t seed, uint64_t shot0, uint64_t nshots,
                                  uint64_t *d_meas, uint64_t *d_det, uint64_t *d_obs, void *cuda_stream);

/*
 * sp_sample_batch -- many programs (uneven sizes, shot counts, seeds) in one
 * enqueue: Algorithm 1 "Sampling" (Eq. sampling) for each program.  Program
 * i samples shots 0..nshots[i]-1 with seeds[i] into d_meas[i], d_det[i],
 * d_obs[i] (the arrays, or any entry, may be NULL).  Records are identical
 * to nprog separate sp_sample calls.
 *   Programs on the fused path are grouped by the launch shape their build-
 *   time autotuner chose (shots per tile, threads, CTAs per SM); each group
 *   runs as one persistent kernel over a list of (program, shot tile) work
 *   items.  The enqueue sequence is captured once in a CUDA graph per plan
 *   = (device, program set, each program's configuration, shot counts) and
 *   replayed: seeds and output pointers are not part of the plan, they are
 *   copied into the plan's device parameter block on cuda_stream before
 *   every launch.  Other programs are sampled through their own path on
 *   cuda_stream after the graph.
 *   Plans are cached per process (at most 8, least recently used dropped);
 *   a plan is dropped when one of its programs is freed or reconfigured
 *   (sp_set_path, sp_set_fused_config, sp_set_chunk).  Dropping a plan waits
 *   for the device.  Calls that share a plan must be ordered by the caller
 *   (same stream, or synchronised): they share its parameter block.
 * Errors: INVALID_ARG (NULL arrays or programs, misaligned outputs, programs
 * of another device), OOM, CUDA.
 */
SP_API sp_status sp_sample_batch(sp_program *const *progs, uint32_t nprog, const uint64_t *seeds,
                          const uint64_t *nshots, uint64_t *const *d_meas,
                          uint64_t *const *d_det, uint64_t *const *d_obs, void *cuda_stream);

/*
 * sp_expect -- analytic detector (then observable) parity expectations
 * E_j = E[(-1)^{D_j}] as log|E_j| in FP32:
 *     log|E_j| = sum_c [channel c touches row j] * log|1 - 2 kappa_c p_c|
 * with kappa = 1 (X/Y/Z_ERROR), 2/3 (DEPOLARIZE1), 8/15 (DEPOLARIZE2): the
 * share of a channel's outcomes with odd overlap with any nonzero mask
 * (Sec. 3.1's channel distributions, applied to the row's affine form).
 * Valid for every p in [0, 1]: a factor is negative above kappa*p = 1/2 and
 * zero at equality, where log|E_j| = -inf (sp_expect_sign gives the sign).
 *   d_p     num_channels FP32 probabilities (random-measurement channels are
 *           ignored), or NULL for the circuit's own probabilities.
 *   d_logE  num_detectors + num_observables FP32 outputs.
 * Errors: INVALID_ARG (NULL prog or d_logE), OOM, CUDA.
 */
SP_API sp_status sp_expect(sp_program *prog, const float *d_p, float *d_logE, void *cuda_stream);

/*
 * sp_expect_sign -- the signs of the expectations of sp_expect:
 *     sign E_j = (-1)^{c_j} * prod_c [channel c touches row j] sign(1 - 2 kappa_c p_c)
 * written as FP32 +1 or -1, and 0 where some factor is exactly zero (then
 * E_j = 0).  c_j is the constant bit of the row (sp_export_rows).
 *   d_p     as in sp_expect;  d_sign  num_detectors + num_observables outputs.
 * Errors: INVALID_ARG (NULL prog or d_sign), OOM, CUDA.
 */
SP_API sp_status sp_expect_sign(sp_program *prog, const float *d_p, float *d_sign, void *cuda_stream);

/*
 * sp_expect_grad -- adjoint of sp_expect:
 *     d_grad_p[c] = sum_j d_grad_logE[j] * d log|E_j| / d p_c
 *                 = -2 kappa_c / (1 - 2 kappa_c p_c) * sum_j A[c,j] g_j
 * (valid on both sides of kappa_c p_c = 1/2; infinite at equality).
 *   d_p, d_grad_logE  inputs (d_p may be NULL as in sp_expect)
 *   d_grad_p          num_channels FP32 outputs (overwritten)
 */
SP_API sp_status sp_expect_grad(sp_program *prog, const float *d_p, const float *d_grad_logE,
                         float *d_grad_p, void *cuda_stream);

/*
 * sp_export_rows -- copy coefficient rows to the host for inspection:
 * which = 0 measurements, 1 detectors, 2 observables.  Row r occupies
 * row_words uint64 words of h_out (bit 0 = constant c_j, bit s = symbol s);
 * row_words must be >= ceil((num_symbols+1)/64).  Synchronous.
 */
SP_API sp_status sp_export_rows(const sp_program *prog, int32_t which, uint64_t *h_out, uint64_t row_words);

/*
 * sp_export_channels -- per-channel threshold T and kind (0 = one symbol
 * Bernoulli, 1 = DEPOLARIZE1, 2 = DEPOLARIZE2, 3 = random measurement) and
 * first symbol.  Arrays of num_channels entries; any may be NULL.
 */
SP_API sp_status sp_export_channels(const sp_program *prog, uint32_t *h_T, uint8_t *h_kind, uint64_t *h_sym0);

/* sp_set_path -- force the sampler variant (SP_PATH_*); AUTO restores the
 * build-time choice. */
SP_API sp_status sp_set_path(sp_program *prog, int32_t path);

/*
 * sp_set_fused_config -- choose the fused kernel variant by hand instead of
 * the build-time autotuner's choice: tile_shots 32, 64 or 128 (shots per
 * CTA tile; 128 = four Philox streams per thread); variant 1 (two CTAs per
 * SM: 512 threads for 32- and 64-shot tiles, 256 threads for 128), 2 (one
 * CTA of 512 threads per SM compiled with more registers; for 32-shot tiles
 * it is the same kernel as 1) or 3 (64-shot tiles only: four CTAs of 256
 * threads per SM).  INVALID_ARG if the tile's records do not fit in shared
 * memory.  Records are identical for every variant.
 */
SP_API sp_status sp_set_fused_config(sp_program *prog, int32_t tile_shots, int32_t variant);

/* sp_set_chunk -- shots per internal chunk (multiple of 1024, 0 = default). */
SP_API sp_status sp_set_chunk(sp_program *prog, uint64_t chunk_shots);

/*
 * sp_set_stream -- choose the definition of the fault draw ("sample b from
 * P_C", Algorithm 1; Sec. 3.1 distributions) used by every later sampling
 * call on this program.  Both give records with the same distribution;
 * their bits differ.
 *   1  (default) per-channel Philox4x32-10: channel c of shot t reads word
 *      c%4 of Philox(counter (t lo, t hi, c/4, 0)), as described above.
 *   2  grouped: random-outcome channel of rank r reads bit r%32 of word
 *      (r/32)%4 of Philox(t lo, t hi, r/128, 3); the other channels, in
 *      order, form groups of 32; group g fires when word g%4 of Philox(t lo,
 *      t hi, g/4, 1) is below floor((1 - prod(1 - p_i)) 2^32); in a group
 *      that fired, channel i reads word i%4 of Philox(t lo, t hi, 8g + i/4,
 *      2) and fires below floor(p_i / (1 - prod_{j>=i}(1 - p_j)) 2^32) while
 *      none before it has (the last channel with p > 0 always), then below
 *      its own floor(p_i 2^32); a depolarizing channel that fired takes
 *      k = min(floor(u m / U), m - 1) with U the threshold that decided it.
 *      About 16x fewer Philox evaluations than stream 1 at p = 1e-3 over
 *      groups of 32 channels; stream 1 stays preferable where channels fire
 *      often.  Runs on the fused path only (the path is set to it);
 *      sp_sample_static and the staged and dense paths draw stream 1.
 * Switching streams re-runs the build's launch-shape autotuner for the new
 * stream (cached per circuit shape), replacing a sp_set_fused_config choice.
 * Errors: INVALID_ARG (stream not 1 or 2; stream 2 without the fused path),
 * OOM, CUDA.
 */
SP_API sp_status sp_set_stream(sp_program *prog, int32_t stream);

/*
 * sp_device_status -- wait for the device, then report and clear the status
 * word that the program's tensor-core kernel sets when one of its bounded
 * waits (on a bulk copy or on its own MMAs) ran out: *status = 0 and SP_OK
 * if every launch since the last call completed; *status = 1 and
 * SP_ERR_TIMEOUT if some tile gave up (its records are then not written).
 * sp_sample_host, which synchronises anyway, returns SP_ERR_TIMEOUT the same
 * way.  Other kernels have no waits and leave the word 0.
 */
SP_API sp_status sp_device_status(sp_program *prog, int32_t *status);

/*
 * sp_set_wait_limit -- bound, in nanoseconds, of the tensor-core kernel's
 * waits for a stage's operands and for the MMAs that free a stage (0 = the
 * default, 2 s).  A wait that runs out makes the tile give up: the kernel
 * stops issuing work, waits for the copies and MMAs already issued (with
 * the fixed 2 s bound), frees its TMEM, records status 1 and returns.
 * Failure-path tests set a bound too short for any stage to be ready.
 */
SP_API sp_status sp_set_wait_limit(sp_program *prog, uint64_t ns);

/* Kernel classes reported by sp_profile_read. */
enum {
    SP_KERNEL_DRAW = 0,      /* Philox fault draw */
    SP_KERNEL_PRODUCT = 1,   /* GF(2) product (sparse or dense variant) */
    SP_KERNEL_EMIT = 2,      /* bit-sliced -> shot-major record transpose */
    SP_KERNEL_FUSED = 3,     /* fused draw + product */
    SP_KERNEL_TENSOR = 4,    /* tensor-core (tcgen05) product */
    SP_KERNEL_CONSTS = 5,    /* per-launch channel-block constants of the fused draw */
    SP_KERNEL_CLASSES = 8
};

/*
 * sp_profile_enable -- when on != 0, every kernel the program launches in
 * sp_sample / sp_sample_host is bracketed by a pair of CUDA events recorded
 * on the launching stream.  sp_profile_read waits for those events, writes
 * the accumulated milliseconds and launch counts per kernel class into
 * ms[SP_KERNEL_CLASSES] and launches[SP_KERNEL_CLASSES] (either may be NULL)
 * and clears the accumulators.
 */
SP_API sp_status sp_profile_enable(sp_program *prog, int32_t on);
SP_API sp_status sp_profile_read(sp_program *prog, double *ms, uint64_t *launches);

/*
 * sp_debug_fail_alloc -- allocation-failure injection for tests of the
 * error paths (host-side: no GPU fault is involved).  After `after` more
 * successful library allocations (device buffers from cudaMalloc, and the
 * host-side program object of sp_build), the next one fails as if the
 * device or host were out of memory and the hook disarms; after < 0
 * disarms it.  The failing call returns SP_ERR_OOM, releases what it had
 * allocated and leaves the program (if any) usable.  No paper counterpart.
 */
SP_API sp_status sp_debug_fail_alloc(int64_t after);

/* sp_debug_live_allocs -- device allocations and programs the library
 * currently holds (either pointer may be NULL); used to check that failing
 * calls leak nothing.  Host only; no paper counterpart. */
SP_API sp_status sp_debug_live_allocs(int64_t *device_allocs, int64_t *host_programs);

/* sp_batch_plans -- number of cached sp_sample_batch plans and the cache's
 * capacity (either pointer may be NULL).  Host only; no paper counterpart
 * (inspection of the batched form's plan cache). */
SP_API sp_status sp_batch_plans(uint32_t *count, uint32_t *capacity);

/* sp_free -- release a program (NULL is allowed). */
SP_API void sp_free(sp_program *prog);

/* sp_last_error -- message of the last failing call on this thread. */
SP_API const char *sp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SYMPHASE_H */
