"""GPU noise generator: bit-identical Philox words with the oracle and with
cuRAND's Philox4_32_10 (a library routine), Box-Muller noise within float32
rounding of the oracle's float64 values."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_11719_gb300 import inputs as I  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def S():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2302_11719_gb300 import smppi
    return smppi


def _ctl(S, **over):
    pr = I.single_problem(**over)
    return S.Controller(pr.params, pr.track), pr


@pytest.mark.parametrize("seed,it,inst", [(0, 0, 0), (0xDEADBEEF12345678, 7, 3),
                                          (2**64 - 1, 2**32 - 1, 2**24 - 1)])
def test_philox_words_bit_identical(S, orc, seed, it, inst):
    ctl, pr = _ctl(S, K=8, T=10, seed=seed)
    K, T = 37, 9
    raw = torch.zeros((K, (T + 1) // 2, 4), dtype=torch.int32, device="cuda")
    S.smppi_debug_noise(ctl.h, it, inst, K, T, None, raw)
    got = raw.cpu().numpy().view(np.uint32)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for k in range(K):
        for p in range((T + 1) // 2):
            assert list(got[k, p]) == orc.philox4x32((k, p, it, inst << 8), key), (k, p)


def test_philox_matches_curand(S):
    so = os.path.join(HERE, "cuda", "_build", "libcurand_probe.so")
    os.makedirs(os.path.dirname(so), exist_ok=True)
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                           "-Xcompiler", "-fPIC", "-o", so,
                           os.path.join(HERE, "cuda", "curand_probe.cu")])
    L = C.CDLL(so)
    L.curand_probe.argtypes = [C.c_uint64, C.c_void_p, C.c_int, C.c_void_p]
    seed = 0x0123456789ABCDEF
    ctl, pr = _ctl(S, K=8, T=10, seed=seed)
    K, T, it, inst = 50, 12, 5, 11
    raw = torch.zeros((K, T // 2, 4), dtype=torch.int32, device="cuda")
    S.smppi_debug_noise(ctl.h, it, inst, K, T, None, raw)
    ctr = np.array([[k, p, it, inst << 8] for k in range(K) for p in range(T // 2)], np.uint32)
    ctr_d = torch.as_tensor(ctr.view(np.int32), device="cuda")
    out = torch.zeros_like(ctr_d)
    assert L.curand_probe(seed, ctr_d.data_ptr(), ctr.shape[0], out.data_ptr()) == 0
    assert np.array_equal(out.cpu().numpy().view(np.uint32).reshape(K, T // 2, 4),
                          raw.cpu().numpy().view(np.uint32))


def test_noise_values_match_oracle(S, orc):
    ctl, pr = _ctl(S, K=8, T=10, seed=42)
    K, T = 300, 51
    eps = torch.zeros((K, T, 2), device="cuda")
    S.smppi_debug_noise(ctl.h, 3, 0, K, T, eps, None)
    m = orc.Model(pr.params, pr.track)
    ref = orc.noise_block(m.with_(seed=42), 3, 0, range(K), T)
    got = eps.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 0.05)) < 2e-6
