"""The dense forms of the product (Eq. sampling as a contraction over every
symbol): the CUDA-core AND/popcount kernel and the tcgen05 tensor-core
kernel (0/1 E4M3 operands, exact FP32 sums, parity), against the CPU oracle
through the C ABI. Records are bit-exact; the tensor kernel's bounded waits
must all have completed (device status 0)."""
import numpy as np
import pytest

import oracle
from workloads import (mirror_circuit, random_clifford_circuit, random_layered, random_small_circuit,
                       repetition_code, surface_code)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2311_03906_gb300 as sp  # noqa: E402

CIRCUITS = {
    "rep5": lambda: repetition_code(5, 5, 0.01),
    "surf5": lambda: surface_code(5, 5, 2e-3),
    "layered40": lambda: random_layered(40, 40, depolarize=0.01, seed=3),
    # 480 record rows (4 row tiles), ~14k symbols (57 K stages of 256)
    "layered120": lambda: random_layered(120, 60, depolarize=0.01, seed=5),
    "rand5": lambda: random_small_circuit(38, 210, seed=905),
    "cliff4": lambda: random_clifford_circuit(14, 240, seed=704),
    # dense rows (about 40 % of the coefficients set), 3,072 symbols
    "mirror48": lambda: mirror_circuit(48, 16, p=0.01, seed=2),
}
PATHS = {"dense": sp.PATH_DENSE, "tensor": sp.PATH_TENSOR}


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def _check(prog, ref, shots, seed, shot0):
    m, d, o = prog.sample(shots, seed=seed, shot0=shot0)
    torch.cuda.synchronize()
    rm, rd, ro = ref.sample(seed, shot0, shots)
    np.testing.assert_array_equal(_u64(m), rm)
    np.testing.assert_array_equal(_u64(d), rd)
    np.testing.assert_array_equal(_u64(o), ro)


@pytest.mark.parametrize("path", list(PATHS))
@pytest.mark.parametrize("name", list(CIRCUITS))
def test_dense_paths_match_oracle(name, path):
    c = CIRCUITS[name]()
    prog, ref = sp.build(c), oracle.Program(c)
    prog.set_path(PATHS[path])
    assert prog.info["path"] == PATHS[path]
    # ragged: not a multiple of 32 or of the 128-shot tensor tile, unaligned start
    _check(prog, ref, 1000, seed=7, shot0=77)
    _check(prog, ref, 33, seed=8, shot0=(1 << 32) - 5)
    assert prog.device_status() == 0


@pytest.mark.parametrize("path", list(PATHS))
def test_dense_paths_equal_fused_on_d11(path):
    """d=11 surface code: 4,096 shots on the dense path equal the fused
    path's records bit for bit; a few shots are recomputed by the oracle."""
    c = surface_code(11, 11, 1e-3)
    prog, ref = sp.build(c), oracle.Program(c)
    fm, fd, fo = prog.sample(4096, seed=21, shot0=1000)
    prog.set_path(PATHS[path])
    m, d, o = prog.sample(4096, seed=21, shot0=1000)
    torch.cuda.synchronize()
    assert prog.device_status() == 0
    for a, b in ((m, fm), (d, fd), (o, fo)):
        np.testing.assert_array_equal(_u64(a), _u64(b))
    pick = np.array([0, 1, 31, 32, 127, 128, 2047, 4095])
    rm, rd, ro = ref.sample_shots(21, 1000 + pick)
    np.testing.assert_array_equal(_u64(m)[pick], rm)
    np.testing.assert_array_equal(_u64(d)[pick], rd)


def test_tensor_path_chunked_equals_unchunked():
    c = random_layered(120, 60, depolarize=0.01, seed=5)
    prog = sp.build(c)
    prog.set_path(sp.PATH_TENSOR)
    m1, d1, o1 = prog.sample(5000, seed=3, shot0=11)
    prog.set_chunk(2048)
    m2, d2, o2 = prog.sample(5000, seed=3, shot0=11)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(_u64(m1), _u64(m2))
    assert prog.device_status() == 0


def test_tensor_path_large_count_equals_fused():
    """700,001 shots from an unaligned start (a ragged last 128-shot tile,
    more than a million-row fault-bit buffer) on the tensor path, twice in
    a row on the same buffers: records equal the fused path's bit for bit,
    and a few shots are recomputed by the oracle."""
    c = mirror_circuit(48, 16, p=0.02, seed=4)
    prog, ref = sp.build(c), oracle.Program(c)
    n, shot0 = 700_001, 12_345
    prog.set_path(sp.PATH_FUSED)
    fm, fd, fo = prog.sample(n, seed=5, shot0=shot0)
    prog.set_path(sp.PATH_TENSOR)
    for _ in range(2):
        m, d, o = prog.sample(n, seed=5, shot0=shot0)
        torch.cuda.synchronize()
        assert prog.device_status() == 0
        for a, b in ((m, fm), (d, fd), (o, fo)):
            assert torch.equal(a, b)
    pick = np.array([0, 1, 127, 128, 350_000, n - 129, n - 128, n - 1])
    rm, rd, ro = ref.sample_shots(5, shot0 + pick)
    np.testing.assert_array_equal(_u64(m)[pick], rm)
    np.testing.assert_array_equal(_u64(d)[pick], rd)


def test_path_choice_is_measured_where_rows_are_dense():
    """Mirror circuits have dense rows: the build times the sparse and both
    dense forms and keeps the fastest; the surface code (0.3 % dense) is
    never probed with the dense forms."""
    dense = sp.build(mirror_circuit(128, 24, p=0.01, seed=3))
    probe = dense.info["path_probe_ms"]
    assert dense.info["density"] > 0.2
    assert probe[sp.PATH_DENSE] > 0 and probe[sp.PATH_TENSOR] > 0
    chosen = dense.info["path"]
    # the default (sparse) form is kept unless another is at least 3 % faster
    assert probe[chosen] > 0 and probe[chosen] <= min(t for t in probe if t > 0) / 0.97 + 1e-9
    sparse = sp.build(surface_code(11, 11, 1e-3))
    assert sparse.info["density"] < 0.01
    assert sparse.info["path_probe_ms"][sp.PATH_DENSE] == 0 and sparse.info["path"] == sp.PATH_FUSED
