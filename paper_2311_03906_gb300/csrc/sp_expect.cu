// sp_expect.cu -- analytic detector-parity expectations and their adjoint.
//
// For a detector (or observable) row D_j = c_j ^ <a_j, s> with independent
// channels, E[(-1)^{D_j}] = (-1)^{c_j} prod_c (1 - 2 P_c(odd)), where
// P_c(odd) is the probability that the channel's drawn symbol bits have odd
// overlap with the row's mask on that channel.  For every nonzero mask this
// is kappa_c * p_c: kappa = 1 for a one-symbol channel, 2/3 for
// DEPOLARIZE1 (2 of its 3 outcomes) and 8/15 for DEPOLARIZE2 (8 of 15).
//   K7 k_expect_fwd   log|E_j| = sum_c inc[j,c] * log(1 - 2 kappa_c p_c)
//   K8 k_expect_bwd   dL/dp_c = -2 kappa_c / (1 - 2 kappa_c p_c) * sum_j inc[j,c] g_j
// inc is the bit-packed target x channel incidence matrix (and its
// transpose for the adjoint), built once by sp_build.
#include <algorithm>

#include "sp_internal.h"

namespace sp {

__global__ void k_channel_weights(const float *__restrict__ p, const float *__restrict__ kappa,
                                  int64_t nch, float *w, float *dw)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nch) return;
    const float k = kappa[c];
    const float x = 2.0f * k * p[c];
    if (w) w[c] = k > 0.f ? log1pf(-x) : 0.f;
    if (dw) dw[c] = k > 0.f ? -2.0f * k / (1.0f - x) : 0.f;
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
sp_status weights(sp_program *P, const float *d_p, bool grad, cudaStream_t s, float **w)
{
    if (!P->d_wbuf) {
        if (cudaMalloc((void **)&P->d_wbuf, (size_t)std::max<int64_t>(P->n_ch, 1) * 2 * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            P->d_wbuf = nullptr;
            return set_error(SP_ERR_OOM, "cudaMalloc of the channel weights failed");
        }
    }
    const float *p = d_p ? d_p : P->d_chP;
    float *wb = P->d_wbuf, *dwb = P->d_wbuf + std::max<int64_t>(P->n_ch, 1);
    if (P->n_ch > 0) {
        k_channel_weights<<<(unsigned)ceil_div(P->n_ch, 256), 256, 0, s>>>(p, P->d_kappa, P->n_ch,
                                                                          grad ? nullptr : wb, grad ? dwb : nullptr);
        SP_CUDA(cudaGetLastError());
    }
    *w = grad ? dwb : wb;
    return SP_OK;
}
}  // namespace

sp_status expect_fwd(sp_program *P, const float *d_p, float *d_logE, cudaStream_t s)
{
    const int64_t ntgt = P->n_det + P->n_obs;
    if (ntgt == 0) return SP_OK;
    float *w;
    sp_status st = weights(P, d_p, false, s, &w);
    if (st != SP_OK) return st;
    k_expect_fwd<<<(unsigned)ceil_div(ntgt, 8), 256, 0, s>>>(P->d_inc, P->incPitch, ntgt, w, d_logE);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

sp_status expect_bwd(sp_program *P, const float *d_p, const float *d_g, float *d_grad, cudaStream_t s)
{
    if (P->n_ch == 0) return SP_OK;
    float *dw;
    sp_status st = weights(P, d_p, true, s, &dw);
    if (st != SP_OK) return st;
    if (P->n_det + P->n_obs == 0) {
        SP_CUDA(cudaMemsetAsync(d_grad, 0, (size_t)P->n_ch * sizeof(float), s));
        return SP_OK;
    }
    k_expect_bwd<<<(unsigned)ceil_div(P->n_ch, 8), 256, 0, s>>>(P->d_incT, P->incTPitch, P->n_ch, d_g, dw, d_grad);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

}  // namespace sp
