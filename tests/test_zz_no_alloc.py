"""The allocation-free energy entry point (gsb_energy_noalloc). It serves
callers that cannot call cudaMalloc: a steady-state loop that must not block
on allocation, or an application whose own allocator owns the device memory.
Its energies must equal the FP64 oracle's (Eq. 1) and gsb_energy's on
consecutive calls that share its fixed scratch array, it must allocate
nothing on the device, and it must reject sizes beyond its fixed limits.
Collected last on purpose, so a failure here comes after every other test has
run; each test also passes alone in a fresh process."""
import numpy as np
import pytest

import oracle as O
from paper_2508_17655_gb300 import gsb, inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_17655_gb300 import build
    build.build()


def _spins(R, N, seed):
    return (np.random.default_rng(seed).integers(0, 2, size=(R, N)) * 2 - 1).astype(np.int8)


def _call(torch, Jd, N, S, stream):
    R = S.shape[0]
    Sd = torch.from_numpy(S).cuda()
    Ed = torch.full((R,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    used0 = gsb.memory_usage()
    gsb.energy_noalloc(Jd.data_ptr(), N, Sd.data_ptr(), R, Ed.data_ptr(), stream=stream)
    torch.cuda.synchronize()
    return Ed.cpu().numpy(), free0 - torch.cuda.mem_get_info()[0], used0 != gsb.memory_usage()


# N = 300: one block of 64 rows x 5; N = 8000 needs 64,000 bytes of shared
# memory per block, past the 48 KiB default (the opt-in branch); R = 9 and 203
# leave ragged replica blocks of 8
@pytest.mark.parametrize("kind,N,R", [("pm1", 300, 203), ("gauss", 300, 203), ("pm1", 8000, 9)])
def test_noalloc_energy_matches_oracle_on_two_calls(kind, N, R):
    torch = pytest.importorskip("torch")
    J = I.sk_pm1(N, 3).astype(np.float32) if kind == "pm1" else I.sk_gauss(N, 3)
    J64 = J.astype(np.float64)
    P = gsb.Problem.dense(J)
    Jd = torch.from_numpy(np.ascontiguousarray(J)).cuda()
    stream = torch.cuda.current_stream()
    for call, seed in enumerate((11, 12)):  # two calls in a row, different spins
        S = _spins(R, N, seed)
        got, grew, lib_alloc = _call(torch, Jd, N, S, stream)
        ref = O.energy(J64, S)
        if kind == "pm1":
            # integer J: exact on every side
            np.testing.assert_array_equal(got, ref)
            np.testing.assert_array_equal(got, P.energy(S))
        else:
            # FP32 coupling sums against FP64: within 1e-5 of the magnitude of
            # the terms, sum_i |s_i| sum_j |J_ij| / 2
            scale = 0.5 * np.abs(J64).sum()
            assert np.max(np.abs(got - ref)) <= 1e-5 * scale
            np.testing.assert_allclose(got, P.energy(S), rtol=0, atol=1e-5 * scale)
        if call == 1:
            # the second call (kernels already loaded) allocates nothing: neither
            # the device's free memory nor the library's own accounting moves
            assert grew == 0
            assert not lib_alloc
    P.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    N, R = 4, 65537
    Jd = torch.zeros((N, N), dtype=torch.float32, device="cuda")
    Sd = torch.ones((R, N), dtype=torch.int8, device="cuda")
    Ed = torch.zeros((R,), dtype=torch.float64, device="cuda")
    with pytest.raises(gsb.GsbError) as e:
        gsb.energy_noalloc(Jd.data_ptr(), N, Sd.data_ptr(), R, Ed.data_ptr())
    assert e.value.status == gsb.EINVAL
    # N past the staged-spin limit is rejected before anything is launched
    with pytest.raises(gsb.GsbError) as e:
        gsb.energy_noalloc(Jd.data_ptr(), 29001, Sd.data_ptr(), 1, Ed.data_ptr())
    assert e.value.status == gsb.EINVAL
