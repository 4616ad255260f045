"""The operand roundings that the GPU contraction tests emulate (tests/helpers.py), pinned on the CPU:
BF16 against PyTorch's float32 -> bfloat16 conversion (to nearest, ties to even), TF32 against its
definition (11 significant bits, to nearest, ties away from zero)."""
import numpy as np
import pytest

from tests.helpers import round_sig, round_tf32


def test_bf16_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.standard_normal(200000) * 10.0 ** rng.integers(-20, 20, 200000),
                        rng.uniform(0.0, 1.0, 100000)]).astype(np.float32)
    # exact ties of the 8-bit significand: the 9th bit set, nothing below it
    ties = (np.arange(1, 4096, dtype=np.uint32) << np.uint32(15)) | np.uint32(0x3F800000) | np.uint32(0x8000)
    x = np.concatenate([x, ties.view(np.float32), -ties.view(np.float32)])
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(round_sig(x.astype(np.float64), 8), want)


def test_tf32_definition():
    rng = np.random.default_rng(12)
    x = (rng.standard_normal(300000) * 10.0 ** rng.integers(-30, 30, 300000)).astype(np.float32)
    r = round_tf32(x)
    u = r.astype(np.float32).view(np.uint32)
    assert np.all(u & np.uint32(0x1FFF) == 0)                                  # 10 stored significand bits
    m, e = np.frexp(x.astype(np.float64))
    ulp = np.ldexp(1.0, e - 11)                                                # of 11 significant bits
    assert np.all(np.abs(r - x) <= 0.5 * ulp * (1 + 1e-12))                    # to nearest
    assert np.array_equal(np.sign(r), np.sign(x))


def test_tf32_ties_go_away_from_zero():
    base = np.array([1.0, 1.5, 3.0, 1000.0], dtype=np.float32).view(np.uint32)
    ties = (base | np.uint32(0x1000)).view(np.float32)                         # exactly half an ulp above
    up = ((base + np.uint32(0x2000))).view(np.float32).astype(np.float64)
    assert np.array_equal(round_tf32(ties), up)
    assert np.array_equal(round_tf32(-ties), -up)
    below = (base | np.uint32(0x0FFF)).view(np.float32)                        # just under half an ulp
    assert np.array_equal(round_tf32(below), base.view(np.float32).astype(np.float64))
