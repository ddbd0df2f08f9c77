// sp_expect.cu -- analytic detector-parity expectations and their adjoint.
//
// For a detector (or observable) row D_j = c_j ^ <a_j, s> with independent
// channels, E[(-1)^{D_j}] = (-1)^{c_j} prod_c (1 - 2 P_c(odd)), where
// P_c(odd) is the probability that the channel's drawn symbol bits have odd
// overlap with the row's mask on that channel.  For every nonzero mask this
// is kappa_c * p_c: kappa = 1 for a one-symbol channel, 2/3 for
// DEPOLARIZE1 (2 of its 3 outcomes) and 8/15 for DEPOLARIZE2 (8 of 15).
// A factor f_c = 1 - 2 kappa_c p_c is negative where kappa_c p_c > 1/2 (an
// X_ERROR above p = 1/2, DEPOLARIZE1 above 3/4) and zero at equality, so the
// kernels keep log|f_c| and the sign apart:
//   K7 k_expect_fwd   log|E_j| = sum_c inc[j,c] * log|f_c|   (-inf where some f_c = 0)
//      k_expect_sign  sign E_j = (-1)^{c_j} prod_c sign f_c  (0 where some f_c = 0)
//   K8 k_expect_bwd   dL/dp_c = -2 kappa_c / f_c * sum_j inc[j,c] g_j
// inc is the bit-packed target x channel incidence matrix (and its
// transpose for the adjoint), built once by sp_build.
#include <algorithm>

#include "sp_internal.h"

namespace sp {

// Per channel: w = log|f|, dw = d log|f| / dp = -2 kappa / f and the sign
// class of f (0: f > 0, 1: f < 0, 2: f = 0).  For x = 2 kappa p below 1/2,
// log1p keeps the small logarithms accurate; from 1/2 up to 2 the difference
// 1 - x is exact in FP32.
__global__ void k_channel_weights(const float *__restrict__ p, const float *__restrict__ kappa,
                                  int64_t nch, float *w, float *dw, uint32_t *cls)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nch) return;
    const float k = kappa[c];
    const float x = 2.0f * k * p[c];
    const float f = 1.0f - x;
    if (w) w[c] = k > 0.f ? (x < 0.5f ? log1pf(-x) : logf(fabsf(f))) : 0.f;
    if (dw) dw[c] = k > 0.f ? -2.0f * k / f : 0.f;
    if (cls) cls[c] = k > 0.f ? (f < 0.f ? 1u : (f == 0.f ? 2u : 0u)) : 0u;
}

// one warp per target row; set bits of the incidence row select weights
__global__ void k_expect_fwd(const uint32_t *__restrict__ inc, int64_t pitch, int64_t ntgt,
                             const float *__restrict__ w, float *out)
{
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= ntgt) return;
    float acc = 0.f;
    for (int64_t q = lane; q < pitch; q += 32) {
        uint32_t m = inc[(size_t)j * pitch + q];
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            acc += w[q * 32 + b];
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[j] = acc;
}

// one warp per target row: parity of its negative factors, any zero factor,
// and the constant c_j (bit 0 of the row's coefficient words)
__global__ void k_expect_sign(const uint32_t *__restrict__ inc, int64_t pitch, int64_t ntgt,
                              const uint32_t *__restrict__ cls, const uint32_t *__restrict__ A, int64_t apitch,
                              int64_t row0, float *out)
{
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= ntgt) return;
    uint32_t neg = 0, zero = 0;
    for (int64_t q = lane; q < pitch; q += 32) {
        uint32_t m = inc[(size_t)j * pitch + q];
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            const uint32_t c = cls[q * 32 + b];
            neg ^= c & 1u;
            zero |= c >> 1;
        }
    }
    neg = __reduce_xor_sync(0xffffffffu, neg);
    zero = __reduce_or_sync(0xffffffffu, zero);
    if (lane == 0) {
        neg ^= A[(size_t)(row0 + j) * apitch] & 1u;
        out[j] = zero ? 0.0f : (neg ? -1.0f : 1.0f);
    }
}

// one warp per channel
__global__ void k_expect_bwd(const uint32_t *__restrict__ incT, int64_t pitch, int64_t nch,
                             const float *__restrict__ g, const float *__restrict__ dw, float *out)
{
    const int lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= nch) return;
    float acc = 0.f;
    for (int64_t q = lane; q < pitch; q += 32) {
        uint32_t m = incT[(size_t)c * pitch + q];
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            acc += g[q * 32 + b];
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[c] = acc * dw[c];
}

namespace {
// Which per-channel quantities k_channel_weights writes.
enum { W_LOG = 0, W_DERIV = 1, W_CLASS = 2 };

sp_status weights(sp_program *P, const float *d_p, int which, cudaStream_t s, float **w)
{
    const int64_t n = std::max<int64_t>(P->n_ch, 1);
    if (!P->d_wbuf) {
        if (dev_alloc((void **)&P->d_wbuf, (size_t)n * 3 * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            P->d_wbuf = nullptr;
            return set_error(SP_ERR_OOM, "cudaMalloc of the channel weights failed");
        }
    }
    const float *p = d_p ? d_p : P->d_chP;
    float *wb = P->d_wbuf, *dwb = P->d_wbuf + n;
    uint32_t *cb = reinterpret_cast<uint32_t *>(P->d_wbuf + 2 * n);
    if (P->n_ch > 0) {
        k_channel_weights<<<(unsigned)ceil_div(P->n_ch, 256), 256, 0, s>>>(
            p, P->d_kappa, P->n_ch, which == W_LOG ? wb : nullptr, which == W_DERIV ? dwb : nullptr,
            which == W_CLASS ? cb : nullptr);
        SP_CUDA(cudaGetLastError());
    }
    *w = which == W_LOG ? wb : which == W_DERIV ? dwb : reinterpret_cast<float *>(cb);
    return SP_OK;
}
}  // namespace

sp_status expect_fwd(sp_program *P, const float *d_p, float *d_logE, cudaStream_t s)
{
    const int64_t ntgt = P->n_det + P->n_obs;
    if (ntgt == 0) return SP_OK;
    float *w;
    sp_status st = weights(P, d_p, W_LOG, s, &w);
    if (st != SP_OK) return st;
    k_expect_fwd<<<(unsigned)ceil_div(ntgt, 8), 256, 0, s>>>(P->d_inc, P->incPitch, ntgt, w, d_logE);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

sp_status expect_bwd(sp_program *P, const float *d_p, const float *d_g, float *d_grad, cudaStream_t s)
{
    if (P->n_ch == 0) return SP_OK;
    float *dw;
    sp_status st = weights(P, d_p, W_DERIV, s, &dw);
    if (st != SP_OK) return st;
    if (P->n_det + P->n_obs == 0) {
        SP_CUDA(cudaMemsetAsync(d_grad, 0, (size_t)P->n_ch * sizeof(float), s));
        return SP_OK;
    }
    k_expect_bwd<<<(unsigned)ceil_div(P->n_ch, 8), 256, 0, s>>>(P->d_incT, P->incTPitch, P->n_ch, d_g, dw, d_grad);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

sp_status expect_sign(sp_program *P, const float *d_p, float *d_sign, cudaStream_t s)
{
    const int64_t ntgt = P->n_det + P->n_obs;
    if (ntgt == 0) return SP_OK;
    float *c;
    sp_status st = weights(P, d_p, W_CLASS, s, &c);
    if (st != SP_OK) return st;
    k_expect_sign<<<(unsigned)ceil_div(ntgt, 8), 256, 0, s>>>(P->d_inc, P->incPitch, ntgt,
                                                             reinterpret_cast<const uint32_t *>(c), P->d_A,
                                                             P->apitch, P->n_meas, d_sign);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

}  // namespace sp
