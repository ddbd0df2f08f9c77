"""Config 5: fitting per-channel noise probabilities to detector statistics.

d = 11, 11 rounds, p_i ~ U(5e-4, 2e-3) for every fault channel; the target
detector rates come from 1e6 shots sampled at p' = p(1 + delta), delta ~
U(-0.2, 0.2); the loss is sum_j (r_j(p) - r^_j)^2 with r_j = (1 - E_j)/2,
differentiated through sp.expect (forward and hand-written backward
kernels). The sampled records are checked against the oracle on sampled
shots, the sampled rates against the analytic ones at p' (5 sigma)."""
import numpy as np
import pytest

import oracle
from workloads import channel_probabilities, perturbed_probabilities, surface_code, with_channel_probabilities

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2311_03906_gb300 as sp  # noqa: E402


def detector_rates(d, ndet: int, chunk: int = 131072):
    """Fraction of shots in which each detector fired, from shot-major packed
    int64 words (on the GPU, in chunks of shots)."""
    counts = torch.zeros(d.shape[1] * 64, dtype=torch.float64, device=d.device)
    shifts = torch.arange(64, device=d.device, dtype=torch.int64)
    for s0 in range(0, d.shape[0], chunk):
        bits = (d[s0:s0 + chunk].unsqueeze(-1) >> shifts) & 1
        counts += bits.sum(0).reshape(-1).double()
    return (counts[:ndet] / d.shape[0]).float()


def test_config5_fit_to_sampled_detector_rates():
    base = surface_code(11, 11, 1e-3)
    p0 = channel_probabilities(base.num_fault_channels, seed=0)
    pt = perturbed_probabilities(p0, seed=1)
    target_circuit = with_channel_probabilities(base, pt)
    prog_t = sp.build(target_circuit)
    prog = sp.build(with_channel_probabilities(base, p0))
    shots = 1_000_000
    _, d, _ = prog_t.sample(shots, seed=11, meas=False, obs=False)
    torch.cuda.synchronize()
    ndet = prog.num_detectors
    # the target records are the sampler's: bit-exact with the oracle on sampled shots
    ref = oracle.Program(target_circuit)
    pick = np.array([0, 1, 777, 123456, shots - 1])
    np.testing.assert_array_equal(d.cpu().numpy().view(np.uint64)[pick], ref.sample_shots(11, pick)[1])
    r_hat = detector_rates(d, ndet)
    # probability vector over all channels (random-measurement channels stay at 1/2)
    _, kind, _ = prog.channels()
    fault = torch.as_tensor(kind != 3, device="cuda")
    base_p = torch.full((prog.num_channels,), 0.5, device="cuda")
    p_t = base_p.clone()
    p_t[fault] = torch.as_tensor(pt, dtype=torch.float32, device="cuda")
    r_t = (1 - torch.exp(prog.expect_raw(p_t)[:ndet].double())) / 2
    sigma = torch.sqrt(r_t * (1 - r_t) / shots)
    assert torch.all(torch.abs(r_hat.double() - r_t) < 5 * sigma + 1e-7)
    # fit log p from p0 with Adam through the autograd Function
    q = torch.log(torch.as_tensor(p0, dtype=torch.float32, device="cuda")).requires_grad_(True)
    opt = torch.optim.Adam([q], lr=0.01)
    losses = []
    for _ in range(100):
        p = base_p.clone()
        p[fault] = torch.exp(q)
        r = (1 - torch.exp(sp.expect(prog, p)[:ndet])) / 2
        loss = ((r - r_hat) ** 2).sum()
        opt.zero_grad()
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])
