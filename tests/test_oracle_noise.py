"""Pins for the oracle's noise (Algorithm 1 GenerateRandomNoise, Eq. (1) eps ~ N(0, Sigma)).

* Philox4x32-10 against cuRAND's host-side PHILOX4_32_10 generator, an
  independent library implementation run on the CPU.  Its output block j is
  Philox(counter = (lo32(j >> 16), hi32(j >> 16), j & 0xFFFF, 0), key = seed).
* The uniform map's exact values, Box-Muller special values and moments.
* bfloat16 rounding against torch's bfloat16 conversion.
"""
import ctypes
import glob
import math
import os

import numpy as np
import pytest

import oracle
from paper_2308_01654_gb300 import scenarios as sc


def _curand():
    cands = []
    for root in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if root:
            cands += sorted(glob.glob(os.path.join(root, "lib64", "libcurand.so*")))
            cands += sorted(glob.glob(os.path.join(root, "targets", "*", "lib", "libcurand.so*")))
    for c in cands:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


def curand_host_philox(seed: int, offset_words: int, n_words: int) -> np.ndarray:
    L = _curand()
    if L is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    assert L.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert L.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert L.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset_words)) == 0
        out = np.zeros(n_words, dtype=np.uint32)
        assert L.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n_words)) == 0
    finally:
        L.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
@pytest.mark.parametrize("block0", [0, 7, 65530, 5 * 65536 + 77, (1 << 48) + 3, (3 << 48) + (9 << 16) + 65531])
def test_philox_matches_curand_host(seed, block0):
    n_blocks = 12
    words = curand_host_philox(seed, 4 * block0, 4 * n_blocks).reshape(n_blocks, 4)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for i in range(n_blocks):
        j = block0 + i
        hi = j >> 16
        ctr = (hi & 0xFFFFFFFF, hi >> 32, j & 0xFFFF, 0)
        np.testing.assert_array_equal(oracle.philox4x32_10(ctr, key), words[i])


def test_philox_counter_word3_changes_output():
    # word 3 of the counter is XORed into the state like word 1; a bijection in each word
    key = (5, 6)
    outs = {tuple(oracle.philox4x32_10((1, 2, 3, w), key)) for w in range(64)}
    assert len(outs) == 64


def test_uniform24_exact_values():
    assert oracle.uniform24(0) == 2.0 ** -24
    assert oracle.uniform24(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert oracle.uniform24(0x80000000) == 0.5 + 2.0 ** -24
    assert oracle.uniform24(0x000000FF) == 2.0 ** -24          # low 8 bits are dropped
    assert oracle.uniform24(0x00000100) == 2.0 ** -24          # (1 | 1) * 2^-24
    assert oracle.uniform24(0x00000200) == 3.0 * 2.0 ** -24    # (2 | 1) * 2^-24
    # symmetric about 1/2: u(w) + u(~w) == 1
    rng = np.random.default_rng(3)
    for w in rng.integers(0, 2 ** 32, 200, dtype=np.uint64):
        w = int(w)
        assert oracle.uniform24(w) + oracle.uniform24(w ^ 0xFFFFFFFF) == 1.0


def test_box_muller_special_values():
    u_r1 = math.exp(-0.5)  # radius sqrt(-2 ln u0) = 1
    z0, z1 = oracle.box_muller(u_r1, 0.0)
    assert z0 == pytest.approx(1.0, abs=1e-15) and z1 == pytest.approx(0.0, abs=1e-15)
    z0, z1 = oracle.box_muller(u_r1, 0.25)
    assert z0 == pytest.approx(0.0, abs=1e-15) and z1 == pytest.approx(1.0, abs=1e-15)
    z0, z1 = oracle.box_muller(u_r1, 0.5)
    assert z0 == pytest.approx(-1.0, abs=1e-15) and z1 == pytest.approx(0.0, abs=1e-15)
    u = math.exp(-2.0)  # radius 2
    z0, z1 = oracle.box_muller(u, 0.125)
    assert z0 == pytest.approx(math.sqrt(2.0), abs=1e-14) and z1 == pytest.approx(math.sqrt(2.0), abs=1e-14)


def test_noise_is_standard_normal():
    scipy_stats = pytest.importorskip("scipy.stats")
    p = sc.default_params(K=4096, T=64, dt=0.05)
    z = oracle.noise(p, 0).reshape(-1, 2)
    n = z.shape[0]
    for c in range(2):
        x = z[:, c]
        assert abs(x.mean()) < 5.0 / math.sqrt(n)
        assert abs(x.var() - 1.0) < 6.0 * math.sqrt(2.0 / n)
        assert abs(scipy_stats.kurtosis(x, fisher=False) - 3.0) < 0.05
        assert scipy_stats.kstest(x, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 5.0 / math.sqrt(n)


def test_noise_counter_layout():
    """z[t][k] uses counter (t//2, k, iter, session); even t words 0,1 and odd t words 2,3."""
    p = sc.default_params(K=5, T=4, dt=0.05)
    p["seed"], p["session"] = 0x1234_5678_9ABC, 77
    z = oracle.noise(p, 9)
    key = (p["seed"] & 0xFFFFFFFF, p["seed"] >> 32)
    for t in range(4):
        for k in range(5):
            w = oracle.philox4x32_10((t // 2, k, 9, 77), key)
            a, b = (w[0], w[1]) if t % 2 == 0 else (w[2], w[3])
            z0, z1 = oracle.box_muller(oracle.uniform24(a), oracle.uniform24(b))
            assert z[t, k, 0] == z0 and z[t, k, 1] == z1


def test_noise_is_independent_of_K_and_depends_on_iter_and_session():
    p8 = sc.default_params(K=8, T=6, dt=0.05)
    p3 = sc.default_params(K=3, T=6, dt=0.05)
    np.testing.assert_array_equal(oracle.noise(p8, 2)[:, :3], oracle.noise(p3, 2))
    assert not np.array_equal(oracle.noise(p8, 2), oracle.noise(p8, 3))
    p8b = dict(p8, session=1)
    assert not np.array_equal(oracle.noise(p8, 2), oracle.noise(p8b, 2))


def test_round_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    vals = np.concatenate([rng.standard_normal(20000), [0.0, 1.0, -1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 6.25]])
    vals = vals.astype(np.float32).astype(np.float64)  # exactly representable in fp32: no double rounding
    ref = torch.from_numpy(vals.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([oracle.round_bf16(v) for v in vals])
    np.testing.assert_array_equal(got, ref)
    assert oracle.round_bf16(1 + 2 ** -8) == 1.0                 # tie -> even
    assert oracle.round_bf16(1 + 3 * 2 ** -8) == 1 + 2 ** -6     # tie -> even


def test_bf16_noise_is_rounded_fp64_noise():
    p = sc.default_params(K=64, T=8, dt=0.05)
    z = oracle.noise(p, 1)
    pb = dict(p, noise_bf16=1)
    zb = oracle.noise(pb, 1)
    np.testing.assert_array_equal(zb, np.vectorize(oracle.round_bf16)(z))
    assert np.max(np.abs(zb - z) / np.maximum(np.abs(z), 1e-30)) <= 2.0 ** -8
