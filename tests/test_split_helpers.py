"""The split-bf16 helper the parity tests give the oracle (J_hi + J_lo, the
matrix the split form's products use), pinned on the CPU: its rounding equals
torch's float32 -> bfloat16 conversion (round to nearest, ties to even) on
random values, exact ties and values that carry into the exponent, and the
split leaves at most 2^-17 |J| (J - J_hi is at most 2^-8 |J|, and rounding it
to bf16's 8 significant bits leaves at most 2^-9 of that)."""
import numpy as np
import pytest

from tests._parity import bf16_rne, bf16_split_sum


def _torch_bf16(a):
    torch = pytest.importorskip("torch")
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy()


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(3)
    vals = [rng.normal(size=20000).astype(np.float32),
            (rng.normal(size=20000) * 1e-30).astype(np.float32),
            (rng.normal(size=20000) * 1e30).astype(np.float32)]
    # exact ties: the 16 discarded bits are 0x8000, kept part odd and even
    base = rng.integers(0, 1 << 7, size=4000, dtype=np.uint32) << 16 | np.uint32(0x3F800000)
    ties = (base | np.uint32(0x8000)).view(np.float32)
    # values whose rounding carries into the exponent (mantissa all ones)
    carry = (np.arange(1, 200, dtype=np.uint32) << 23 | np.uint32(0x7FFFFF)).view(np.float32)
    for a in vals + [ties, -ties, carry, -carry]:
        np.testing.assert_array_equal(bf16_rne(a), _torch_bf16(a))


def test_split_residue_bound():
    rng = np.random.default_rng(4)
    J = (rng.normal(size=(300, 300)) / np.sqrt(300)).astype(np.float32)
    S = bf16_split_sum(J)
    J64 = J.astype(np.float64)
    assert np.all(np.abs(S - J64) <= 2.0 ** -17 * np.abs(J64))
    # and the split is not the identity: the residue is there
    assert np.any(S != J64)
